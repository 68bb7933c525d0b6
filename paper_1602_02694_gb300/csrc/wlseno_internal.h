// Internal declarations of libwlseno (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/wlseno.h"

// The pointer qualifier of the per-cell kernel bodies (k_recon_tpc*.cuh,
// k_reconstruct.cuh, k_flux_cell.cuh): __restrict__, except in the
// persistent step kernel, whose phases read arrays that earlier phases of
// the same launch wrote (there the loads must stay coherent).
#ifndef WLSENO_BODY_RESTRICT
#define WLSENO_BODY_RESTRICT __restrict__
#endif

namespace wlseno {

constexpr int kMaxDim = 3;
constexpr int kMaxM = 10;        // Taylor coefficients the kernels are built for
constexpr int kMaxQ = 3;         // quadrature points per facet
constexpr int kMaxFacets = 4;    // facets per simplex

// Quadrature points per facet: the vertex (1-D), two Gauss-Legendre points
// on an edge (2-D), the three-point degree-2 rule on a triangle (3-D).
__host__ __device__ constexpr int nq_of(int dim) { return dim == 1 ? 1 : dim == 2 ? 2 : 3; }

// Host-side result of the mesh / stencil setup (host_mesh.cpp).
struct HostSetup {
  int dim = 0, p = 0, m = 0, nq = 0, n_meshes = 0;
  int64_t N = 0, nnz = 0;
  int max_n = 0, min_n = 0;
  std::vector<int64_t> row_ptr;   // [N+1]
  std::vector<int64_t> cols;      // [nnz], centre first, then increasing index
  std::vector<double> coords;     // [N][dim+1][dim] unwrapped vertices
  std::vector<double> centroid;   // [N][dim]
  std::vector<double> volume;     // [N]
  std::vector<double> h;          // [N] mean edge length
  std::vector<double> inradius;   // [N]
  std::vector<int32_t> mesh_of;   // [N]
  std::vector<double> period;     // [n_meshes][3]
  std::vector<double> rmin;       // [n_meshes] smallest inradius
  std::vector<int32_t> nbr;       // [N][dim+1]: (j << 2) | f' or -1 (boundary)
  std::vector<double> fgeo;       // [N][dim+1][4]: owner's unit normal (dim), area
  std::vector<double> fpts;       // [N][dim+1][nq][dim]: (x_q - x_i) / h_i
  // transposed stencils (adjoint gather): for cell j, the ELL slots t*N + c
  // with stencil row t >= 1 of cell c equal to j, ordered by (c, t)
  std::vector<int64_t> tr_ptr;    // [N+1]
  std::vector<int64_t> tr_slot;   // [nnz - N]
  // balanced-stencil candidates (when asked for): the cells of the enlarged
  // ring of each cell, centre excluded, ascending
  std::vector<int64_t> bal_ptr;   // [N+1]
  std::vector<int64_t> bal_idx;
};

// new_to_old order of one mesh's cells along the Hilbert curve of their
// centroids (reorder.cpp); false on a bad vertex index.
bool hilbert_order(const wlseno_mesh& m, std::vector<int64_t>* new_to_old);

// balance_steps > 0 also collects, for every cell, the cells within that
// many vertex-sharing steps (the balanced-stencil candidates).
wlseno_status build_host_setup(const wlseno_mesh* meshes, int n_meshes,
                               const wlseno_stencil_opts* opts, HostSetup* out,
                               std::string* err, int balance_steps = 0);

// ---------------------------------------------------------------------------
// device-side views handed to the kernel launchers
// ---------------------------------------------------------------------------
// Per-facet coefficients of the FP32-bulk scalar flux, in the orientation of
// the facet's lower-indexed cell (identical in both cells' records): the
// reference coefficient (Burgers: |f| (n_1+..+n_d)/2, advection: |f| v.n) as
// a double-float pair (hi + lo), the FP32 normal factor (Burgers:
// n_1+..+n_d, advection: v.n) and the FP32 facet measure |f|.
struct FacetF32 {
  float pref_hi, pref_lo;
  float coef;
  float area;
};

struct DeviceMesh {
  int dim, p, m, nq;
  int64_t N, nnz;
  const int32_t* st_ptr;    // [N+1]
  const int32_t* st_idx;    // [nnz]
  const double* coords;     // [N][dim+1][dim]
  const double* centroid;   // [N][dim]
  const double* h;          // [N]
  const double* volume;     // [N]
  const double* inv_volume; // [N] 1 / volume
  const double* inradius;   // [N]
  const int32_t* mesh_of;   // [N]
  const double* period;     // [n_meshes][3]
  const int32_t* nbr;       // [N][dim+1]
  const double* fgeo;       // [N][dim+1][4]
  const double* fpts;       // [N][dim+1][nq][dim]
  const float* fpts32;      // same, FP32
  double* A64;              // [nnz][m]
  float* A32;               // [nnz][m]
  // ELL copies for the thread-per-cell kernel: row t of cell i at t*N + i
  int nmax;                 // largest stencil
  int32_t* st_ell;          // [nmax][N]
  double* A64e;             // [nmax][m][N]
  // FP32 row records of the staged thread-per-cell kernel: record (t, i) at
  // (t*N + i)*rec_width floats holds the m moments of row t of cell i, then
  // the stencil index (int32 bits), then zero padding to a 16-byte multiple
  float* rec32;             // [nmax][N][rec_width]
  // FP32 row geometry for the moments-on-the-fly kernel (FP32-bulk): record
  // (t, i) at (t*N + i)*4 floats holds (x_j - x_i)/h_i (dim floats, minimum
  // image), the stencil index as int32 bits, zeros; own32 holds every cell's
  // own central moments of degree >= 2 in absolute units (own_width floats)
  float* geo32;             // [nmax][N][4]
  float* own32;             // [N][own_width]
  int own_width;            // own32_width(dim, m)
  const FacetF32* ff32;     // [N][dim+1] FP32-bulk scalar flux coefficients (else null)
  const float2* inv_vol2;   // [N] FP32-bulk scalar and 2-D Euler: 1/|tau| as a double-float pair (else null)
  const float4* nf32;       // [N][dim+1] FP32-bulk 2-D Euler: owner normal (x, y, 0) and area (else null)
  // [N] FP32-bulk: (eps h_i^2, 1/h_i), each computed in FP64 and rounded to
  // FP32 on the host, so the FP32 kernels need no FP64 arithmetic (else null)
  const float2* hscale32;
  int rec_width;            // round_up(m + 1, 4)
  // the context's non-finite status word: mapped pinned host memory that a
  // kernel sets to 1 when it writes a non-finite value (may be null)
  unsigned int* nf_latch;
};

// Device counters of a context: flagged, rank deficient, nonfinite,
// positivity fallbacks, balanced re-selections.
constexpr int kCounters = 5;

#ifdef __CUDACC__
// A non-finite output: counted for the call's diagnostics and latched in the
// host-visible status word, which the next entry point reports.
__device__ __forceinline__ void report_nonfinite(const DeviceMesh& dm, unsigned long long* counters) {
  atomicAdd(&counters[2], 1ull);
  if (dm.nf_latch) {
    *reinterpret_cast<volatile unsigned int*>(dm.nf_latch) = 1u;
    __threadfence_system();
  }
}
#endif

// Width in floats of one FP32 row record (moments + index, 16-byte padded).
__host__ __device__ constexpr int rec32_width(int m) { return (m + 1 + 3) / 4 * 4; }
// Width in floats of a cell's own-moment record: the m - 1 - dim Taylor
// columns of degree >= 2, 16-byte padded.
__host__ __device__ constexpr int own32_width(int dim, int m) { return (m - 1 - dim + 3) / 4 * 4; }

struct SchemeParams {
  int pde;
  double vel[3];
  double eps, alpha_c, rank_tol, kappa_flag;
  double gamma;             // Euler: ratio of specific heats
  float alpha_c32;          // alpha_c rounded to FP32 on the host (FP32-bulk weights)
};

// Euler (k_euler.cu): fvals/u/out are [4][N]-major per component.
cudaError_t launch_euler_positivity(const DeviceMesh& dm, double gamma, const double* ubar,
                                    double* fvals, unsigned long long* counters, cudaStream_t s);
cudaError_t launch_euler_flux_stage(const DeviceMesh& dm, double gamma, int precision,
                                    const double* fvals, const double* u, const double* u0,
                                    double a, double b, const double* dt_mesh, bool residual_only,
                                    double* out, unsigned long long* counters, cudaStream_t s);
// Characteristic-wise reconstruction of all four components' facet values.
cudaError_t launch_euler_char(const DeviceMesh& dm, const SchemeParams& sp, int precision,
                              const double* ubar, double* fvals, unsigned long long* counters,
                              cudaStream_t s);
cudaError_t launch_euler_speed(const DeviceMesh& dm, double gamma, const double* ubar,
                               unsigned long long* lmax_bits, int n_meshes, cudaStream_t s);
// FP32-bulk 2-D Euler (k_euler32.cu): out = a u0 + b (u + dt L(u)) (or L(u))
// from the FP32 traces [N][6][4] of the all-components reconstruction
// (TraceOut) and the interleaved pairs pin / p0 ([N][4]) of u and u0; pout
// (may be null) receives the pairs of out.
cudaError_t launch_euler2_flux32(const DeviceMesh& dm, double gamma, const float* traces, const float2* pin,
                                 const float2* p0, double a, double b, const float2* dt2, bool residual_only,
                                 double* out, unsigned long long* counters, float2* pout, cudaStream_t s);
// The interleaved FP32 pairs of the 2-D Euler state and, in the same pass,
// the largest |u| + c per mesh (FP32, as double bits) for the CFL step.
cudaError_t launch_euler2_speed_pairs32(const DeviceMesh& dm, double gamma, const double* u,
                                        unsigned long long* lmax_bits, int n_meshes, float2* pairs,
                                        cudaStream_t s);
// pairs[i][c] = FP32 pair of u[c][i] (the four components of 2-D Euler).
cudaError_t launch_euler2_split_pairs(const double* u, float2* pairs, int64_t N, cudaStream_t s);

// All-components (FP32-bulk 2-D Euler) contexts: the facet values travel as
// FP32 traces of the C = dim + 2 components together, base[(i NP + pt) C + c]
// = hi + (lo + dev) of component c at point pt of cell i, or hi + lo for
// every component where the cell's positivity flag is down (the
// reconstruction writes them; its follow-ups update the components they
// redo, in cells whose flag is up).
struct TraceOut {
  float* base = nullptr;                // [N][NP][C], or null: no traces
  const float2* upair = nullptr;        // [N][C] pairs of the averages
  const unsigned char* pos_ok = nullptr;  // [N]
};

struct ReconOut {
  double* coeffs;           // [N][m] or null
  double* fvals;            // [N][dim+1][nq] facet values, or null when fdev is set
  unsigned long long* counters;  // [4]: flagged, rank deficient, nonfinite, positivity fallbacks
  // FP32-bulk flux path: the facet values as FP32 deviations from the cell
  // average, value = ubar_i + fdev (written instead of fvals when set)
  float* fdev = nullptr;    // [N][dim+1][nq]
};

// Balanced-stencil re-selection (k_balance.cu).
struct BalanceWork {
  const int32_t* cand_ptr;   // [N+1]
  const int32_t* cand_idx;   // enlarged-ring candidates, centre excluded, ascending
  unsigned long long* state; // [1 + 2 n_meshes]: list length, then per mesh the
                             // order keys of max u and of max -u
  int* list;                 // [N] cells out of range
  unsigned long long* count; // cells re-solved on a balanced stencil (accumulated)
  double margin;             // out of range: beyond [min, max] by margin * range of u
  int n_meshes;
};
// Range test and re-selection on the output of a reconstruction of ubar;
// overwrites the outputs of the re-solved cells.  *launches = kernels run.
cudaError_t launch_balance(const DeviceMesh& dm, const SchemeParams& sp, const BalanceWork& bw,
                           const double* ubar, const ReconOut& out, cudaStream_t s, int* launches);

// Launchers (return the CUDA error of the launch).
cudaError_t launch_moments(const DeviceMesh& dm, cudaStream_t s);
// Copies the CSR stencil and moments into the ELL arrays.
cudaError_t launch_ell_copy(const DeviceMesh& dm, cudaStream_t s);

// Work lists of the thread-per-cell kernels.  Flagged cells go either to the
// pivoted lane-group path (group_list) or, in FP32-bulk when only moderately
// ill-conditioned, to the thread-level FP64-residual refinement, which reuses
// the FP32 factor the main kernel leaves in one refine record per cell.
struct TpcWork {
  int* group_list;          // [N]
  int* counts;              // [2]: lengths of group_list and of the refine records
  float* refine_buf;        // [N][refine_record_floats(m)] (FP32-bulk contexts; else null)
  // FP32-bulk input: ubar split into FP32 pairs (hi, lo), hi = fl32(ubar),
  // lo = fl32(ubar - hi), so ubar_j - ubar_i = (hi_j - hi_i) + (lo_j - lo_i)
  // to FP32 accuracy without FP64 arithmetic (required when refine_buf is set)
  const float2* upair;      // [N]
  // optional side stream: the pivoted-path kernel runs there, concurrently
  // with the refinement sweep (fork and join through the two events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // FP32-bulk main kernel: form each moment row from geo32/own32 instead of
  // streaming the stored row records
  bool otf = false;
  // entries the group list and the refine records hold (N, or C N when the
  // components of a multi-component context are reconstructed together)
  int64_t capacity = 0;
  // multi-component (2-D Euler, FP32-bulk) kernel: the per-cell positivity
  // flags it writes (1: the traces are used, 0: the averages) and gamma;
  // when set, the facet outputs (ReconOut::fdev) are the traces of TraceOut
  unsigned char* pos_ok = nullptr;
  float gamma = 0.0f;
};

// pair[k] = (fl32(u[k]), fl32(u[k] - fl32(u[k]))) for k < n.
cudaError_t launch_split_pairs(const double* u, float2* pair, int64_t n, cudaStream_t s);

// One refine record (16-byte aligned, read with 16-byte loads): cell index,
// first CSR row and row count (as int32), the centre weight w_c, then the
// solution x (m), D (m), the strict upper triangle of U (m(m-1)/2), eps h^2
// and ubar_i (its FP64 bits as two words, low then high), zero padded.
__host__ __device__ constexpr int refine_record_eps(int m) { return 4 + 2 * m + m * (m - 1) / 2; }
__host__ __device__ constexpr int refine_record_floats(int m) {
  return (refine_record_eps(m) + 3 + 3) / 4 * 4;
}

// Thread-per-cell reconstruction: the main kernel, then the follow-ups on
// the cells it lists (*launches receives their number).
template <typename T, int DIM, int M>
cudaError_t launch_recon_tpc_inst(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                                  const ReconOut& out, const TpcWork& work, cudaStream_t s);
template <typename T, int DIM, int M>
cudaError_t launch_recon_fixup_inst(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                                    const ReconOut& out, const TpcWork& work, cudaStream_t s,
                                    int* launches);
#define WLSENO_DECLARE_TPC(T, D, M)                                                              \
  template <>                                                                                     \
  cudaError_t launch_recon_tpc_inst<T, D, M>(const DeviceMesh&, const SchemeParams&,              \
                                             const double*, const ReconOut&, const TpcWork&,      \
                                             cudaStream_t);                                       \
  template <>                                                                                     \
  cudaError_t launch_recon_fixup_inst<T, D, M>(const DeviceMesh&, const SchemeParams&,            \
                                               const double*, const ReconOut&, const TpcWork&,    \
                                               cudaStream_t, int*);
WLSENO_DECLARE_TPC(double, 1, 3)
WLSENO_DECLARE_TPC(double, 1, 5)
WLSENO_DECLARE_TPC(float, 1, 3)
WLSENO_DECLARE_TPC(float, 1, 5)
WLSENO_DECLARE_TPC(double, 2, 6)
WLSENO_DECLARE_TPC(double, 2, 10)
WLSENO_DECLARE_TPC(double, 3, 10)
WLSENO_DECLARE_TPC(float, 2, 6)
WLSENO_DECLARE_TPC(float, 2, 10)
WLSENO_DECLARE_TPC(float, 3, 10)
#undef WLSENO_DECLARE_TPC

// FP32-bulk 2-D Euler, p = 3: the main kernel for all four components at once
// (one thread per (cell, component), the state pairs work.upair interleaved
// [N][4], ubar the [4][N] state) with the positivity flags work.pos_ok and
// the traces [N][6][4] in out.fdev (TraceOut); the flagged (component, cell)
// pairs are finished by launch_recon_fixup_inst<float, 2, 6> on the same
// outputs.
cudaError_t launch_recon_euler2d(const DeviceMesh& dm, const SchemeParams& sp, const double* ubar,
                                 const ReconOut& out, const TpcWork& work, cudaStream_t s);

// Reconstruction for one component; one translation unit per (T, DIM, M).
template <typename T, int DIM, int M>
cudaError_t launch_reconstruct_inst(const DeviceMesh& dm, const SchemeParams& sp, int G, int R,
                                    const double* ubar, const ReconOut& out, cudaStream_t s);
#define WLSENO_DECLARE_RECON(T, D, M)                                                      \
  template <>                                                                               \
  cudaError_t launch_reconstruct_inst<T, D, M>(const DeviceMesh&, const SchemeParams&, int, \
                                               int, const double*, const ReconOut&,        \
                                               cudaStream_t);
WLSENO_DECLARE_RECON(double, 1, 3)
WLSENO_DECLARE_RECON(double, 1, 5)
WLSENO_DECLARE_RECON(float, 1, 3)
WLSENO_DECLARE_RECON(float, 1, 5)
WLSENO_DECLARE_RECON(double, 2, 6)
WLSENO_DECLARE_RECON(double, 2, 10)
WLSENO_DECLARE_RECON(double, 3, 10)
WLSENO_DECLARE_RECON(float, 2, 6)
WLSENO_DECLARE_RECON(float, 2, 10)
WLSENO_DECLARE_RECON(float, 3, 10)
#undef WLSENO_DECLARE_RECON

// Per-cell flux gather + RK stage: out = a*u0 + b*(u + dt*L(u)); with
// residual_only the output is L(u) itself.
// fdev (FP32-bulk, scalar equations) replaces fvals when set.
// With fdev, pin (the FP32 pairs of u, may be null) gives the jumps between
// cell averages without FP64 arithmetic, and pout (may be null) receives the
// pairs of the written state.  With fdev and pin, and p0 (the pairs of u0)
// unless a = 0 or residual_only, the flux, residual and stage run in
// double-float arithmetic (dfloat.cuh); otherwise in FP64.
cudaError_t launch_flux_stage_impl(const DeviceMesh& dm, const SchemeParams& sp, int precision,
                                   const double* fvals, const float* fdev, const double* u,
                                   const double* u0, double a, double b, const double* dt_mesh,
                                   bool residual_only, double* out, unsigned long long* counters,
                                   cudaStream_t s, const float2* pin = nullptr, float2* pout = nullptr,
                                   const float2* p0 = nullptr, const float2* dt2 = nullptr);
// dt_mesh[k] = cfl * rmin[k] / lambda_max(mesh k), or dt_fixed when > 0;
// dt2 (may be null) receives their double-float pairs, pairs_out (may be
// null) the FP32 pairs of u (made in the wave-speed pass when there is one).
cudaError_t launch_cfl_dt_impl(const DeviceMesh& dm, const SchemeParams& sp, int n_meshes,
                               const double* u, const double* rmin, double cfl, double dt_fixed,
                               unsigned long long* lmax_bits, double* dt_mesh, cudaStream_t s,
                               int* launches, float2* dt2 = nullptr, float2* pairs_out = nullptr);

// One TVD-RK3 step of the scalar equations as one persistent cooperative
// kernel (k_persistent.cu): 2-D meshes, p = 3 or 4 (m = 6, 10), the
// thread-per-cell reconstruction.
struct PersistLaunch {
  DeviceMesh dm;
  SchemeParams sp;
  bool fp32 = false, otf = false;
  double* u = nullptr;             // [N] state, in/out
  double* k1 = nullptr;            // [N] stage states
  double* k2 = nullptr;
  float2* pairs = nullptr;         // [3][N] FP32 pairs of u, k1, k2 (FP32-bulk)
  double* fvals = nullptr;         // [N][NP] (FP64)
  float* fdev = nullptr;           // [N][NP] (FP32-bulk)
  unsigned long long* counters = nullptr;
  int* group_list = nullptr;
  int* counts = nullptr;           // [6]
  float* refine_buf = nullptr;
  int64_t capacity = 0;
  int dt_mode = 0;                 // 0: CFL, 1: dt_fixed, 2: the per-mesh steps in dt_mesh
  double cfl = 0.0, dt_fixed = 0.0;
  double adv_speed = 0.0;          // advection |a|
  int n_meshes = 1;
  const double* rmin = nullptr;
  unsigned long long* lmax = nullptr;
  double* dt_mesh = nullptr;
  float2* dt2 = nullptr;
  unsigned int* sync_words = nullptr;  // [3]: barrier arrivals, generation, status
  unsigned int* timeout_word = nullptr;  // host-visible (mapped) timeout word
  long long spin_cap = 0;
  double flag = 0.0, pivot = 0.0;
};
bool persistent_supported(int dim, int m);
cudaError_t launch_persistent_step(const PersistLaunch& L, cudaStream_t s);
// The flag and pivot thresholds of the thread-per-cell reconstruction.
void tpc_thresholds(const SchemeParams& sp, bool f32, double* flag, double* pivot);

// Work arrays of the adjoint (k_adjoint.cu).
struct AdjointWork {
  double* gfv;             // [N][dim+1][nq] cotangents of each cell's facet traces
  double* contrib;         // [nmax][N] per-(row, cell) cotangents for stencil cells
  double* selfbar;         // [N]
  int* amin_cell;          // [N] facet neighbour giving the centre's beta
  double* amin_val;        // [N]
  const int64_t* tr_ptr;   // [N+1] transposed stencils
  const int64_t* tr_slot;  // [nnz-N]
};
// out = J_L(state)^T lambda (fvals: the facet traces of `state`).
cudaError_t launch_operator_vjp(const DeviceMesh& dm, const SchemeParams& sp, const double* state,
                                const double* fvals, const double* lambda, const AdjointWork& w,
                                double* out, cudaStream_t s, int* launches);
// out = ca x + cb y + cc w + cz dt_mesh z (null inputs skipped).
cudaError_t launch_adj_combine(const DeviceMesh& dm, const double* dt_mesh, const double* x,
                               double ca, const double* y, double cb, const double* w, double cc,
                               const double* z, double cz, double* out, cudaStream_t s);

// Read-only view of a context and launch helpers for entry points that live
// outside capi.cpp (they count launches like the context's own calls).
struct CtxView {
  int device;
  int precision;
  int n_comp;
  bool ready;              // stencils built and moments precomputed
  DeviceMesh dm;
  SchemeParams sp;
  unsigned long long* counters;
  const double* dt;
  bool dev_facets;         // scalar residuals pass facet values as FP32 deviations
};
bool ctx_view(const wlseno_ctx* ctx, CtxView* out);
void ctx_set_error(wlseno_ctx* ctx, const std::string& msg);
cudaError_t ctx_launch_reconstruct(wlseno_ctx* ctx, const double* ubar, const ReconOut& out,
                                   cudaStream_t s);
cudaError_t ctx_launch_flux_residual(wlseno_ctx* ctx, const double* fvals, const float* fdev,
                                     const double* ubar, double* residual, cudaStream_t s);

}  // namespace wlseno
