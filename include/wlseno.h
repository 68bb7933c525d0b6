/*
 * wlseno.h -- C ABI of the GB300 (sm_103a) WLS-ENO finite-volume hot path.
 *
 * Method: Liu & Jiao, "WLS-ENO: Weighted-Least-Squares Based Essentially
 * Non-Oscillatory Schemes for Finite Volume Methods on Unstructured Meshes",
 * arXiv 1602.02694.  Given the cell averages ubar_i of a conserved quantity on
 * a simplex mesh (Sec. 1, Eq. (reconstruction)), every call below works on
 * the cells' WLS-ENO reconstructions of degree p-1 (Sec. 3), the
 * Lax-Friedrichs numerical flux through their facets (Sec. 1, Eq. (flux)),
 * the finite-volume residual (Sec. 1, Eq. (fvm)) and TVD Runge-Kutta 3
 * (Sec. 4.2.1, Eq. (3rd-order-Runge-Kutta)).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a wlseno_status; nothing aborts and no C++ exception
 *    crosses the ABI.  wlseno_status_string() names a status.
 *  - Cell order: cell c of mesh k is global cell (sum of n_cells of meshes
 *    0..k-1) + c, in the caller's order unless wlseno_build_stencils was
 *    asked to reorder (then in the library's order, which perm_out gives).
 *    Per-cell arrays are component-major: [n_comp][n_cells_total] float64.
 *  - Array arguments marked "host or device" may be either: device pointers
 *    are used in place (stream-ordered on `stream`, asynchronous); host
 *    pointers are copied to and from the device inside the call, which then
 *    synchronises `stream` before returning.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - The context owns every derived array (geometry, stencils, moments,
 *    workspace).  Caller buffers are never retained after a call returns (or,
 *    for device pointers, after the stream work it enqueued completes).
 *  - A context is not thread safe; use one context per host thread.
 *  - Non-finite results: a kernel that writes a non-finite cell average,
 *    facet value or residual sets the context's status word (host memory the
 *    device writes).  The next wlseno_reconstruct, wlseno_flux_residual,
 *    wlseno_rk_step or wlseno_step_adjoint on the context returns
 *    WLSENO_ERR_NUMERIC without doing any work and clears the word; a call
 *    that synchronises (host arrays, or rk_step with dt_out) also checks it
 *    after its own work and returns WLSENO_ERR_NUMERIC then.  With device
 *    arrays the report comes once that work has run: at a later call, or
 *    at the first call after a synchronisation.
 */
#ifndef WLSENO_H
#define WLSENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WLSENO_OK = 0,
  WLSENO_ERR_INVALID_ARG = -1, /* null pointer, bad size or option            */
  WLSENO_ERR_MESH = -2,        /* inverted cell, non-manifold or bad facet    */
  WLSENO_ERR_STENCIL = -3,     /* stencil too small (< m cells) or too large  */
  WLSENO_ERR_CUDA = -4,        /* a CUDA runtime call failed                  */
  WLSENO_ERR_OOM = -5,         /* device or host allocation failed            */
  WLSENO_ERR_NUMERIC = -6,     /* non-finite value produced by the kernels    */
  WLSENO_ERR_TIMEOUT = -7,     /* a bounded device wait gave up               */
  WLSENO_ERR_STATE = -8        /* calls made in the wrong order               */
} wlseno_status;

enum { WLSENO_ADVECTION = 0, WLSENO_BURGERS = 1, WLSENO_EULER = 2 };
enum { WLSENO_FP64 = 0, WLSENO_FP32_BULK = 1 };

typedef struct wlseno_ctx wlseno_ctx; /* opaque */

/* One conforming simplex mesh (segments in 1-D, triangles in 2-D,
 * tetrahedra in 3-D).
 * vertices: host [n_vertices][dim] float64.
 * cells:    host [n_cells][dim+1] int64 vertex indices, positively oriented.
 * period:   host [dim]; period[a] > 0 makes axis a periodic with that length
 *           (cells and stencils are unwrapped to their minimum image),
 *           0 makes it transmissive (boundary facets use u+ = u-). */
typedef struct {
  int dim;
  int64_t n_vertices;
  int64_t n_cells;
  const double* vertices;
  const int64_t* cells;
  const double* period;
} wlseno_mesh;

/* Stencil selection (Sec. 3.2).
 * order_p:    p; the reconstruction has degree p-1 and m = C(p-1+dim, dim)
 *             Taylor coefficients.  Supported: 1-D p in {3,5}; 2-D p in {3,4};
 *             3-D p = 3.
 * ring:       k-ring size in the paper's increments (1-D: whole numbers, the
 *             k-ring is 2k+1 cells; 2-D: multiples of 1/2, 1/2 =
 *             facet-sharing, 1 = vertex-sharing; 3-D: multiples of 1/3,
 *             1/3 = face-, 2/3 = edge-, 1 = vertex-sharing).
 * radius_cut: > 0 adds the cells of the next whole ring whose centroid lies
 *             within radius_cut * h_i of the centre cell's centroid.
 * min_rows:   grow stencils (by facet-neighbour increments) until they have at
 *             least this many cells; 0 means ceil(1.5 m).
 * lanes_per_cell, rows_per_lane: shape of the reconstruction kernel: (1,0)
 *             one thread per cell (stencils of at most 64 cells; the default
 *             for 0, 0), or a group of lanes_per_cell lanes of a warp per cell,
 *             each lane holding rows_per_lane stencil rows: (8,2) (8,3) (8,5)
 *             (16,3) (16,4).  wlseno_autotune picks the fastest that fits.
 * moments_mode: FP32-bulk thread-per-cell kernel only (else 0): 0 streams
 *             each stencil row's stored FP32 moments (48 bytes per row for
 *             m = 10); 1 forms them on the fly from the offset
 *             (x_j - x_i)/h_i of the row's cell (16 bytes per row) and that
 *             cell's own central moments (gathered, 16 or 32 bytes per cell)
 *             by the binomial expansion of the Taylor monomials about x_j:
 *             a third of the row bytes for about 40 more FP32 operations per
 *             row.  wlseno_autotune also tries both.
 * reorder:    0 keeps the caller's cell order; 1 renumbers the cells of
 *             every mesh along the Hilbert curve of their centroids (ties by
 *             the caller's index), so that stencil neighbours get nearby
 *             indices and the kernels' gathers stay local for any input
 *             order.  All per-cell arrays of later calls are then in the new
 *             order (see perm_out of wlseno_build_stencils).
 * persistent: 0 runs each RK step as one kernel per phase (captured as a
 *             CUDA graph); 1 runs it as ONE persistent cooperative kernel
 *             whose resident blocks walk the cells of all meshes of the
 *             context through every phase of the step (time step,
 *             reconstruction, follow-ups on flagged cells, flux and stage
 *             update, three stages) with grid-wide barriers in between.
 *             Every barrier wait is bounded (wlseno_set_wait_limit); a wait
 *             that gives up makes the next call return WLSENO_ERR_TIMEOUT.
 *             Scalar equations on 2-D meshes, p = 3 or 4, fixed stencils,
 *             the thread-per-cell shape; else INVALID_ARG.  The results
 *             equal those of persistent = 0 bit for bit. */
typedef struct {
  int order_p;
  double ring;
  double radius_cut;
  int min_rows;
  int lanes_per_cell;
  int rows_per_lane;
  int moments_mode;
  int reorder;
  int persistent;
} wlseno_stencil_opts;

/* Scheme parameters.
 * pde:        WLSENO_ADVECTION (F = a u), WLSENO_BURGERS (F = u^2/2 (1,..,1)),
 *             WLSENO_EULER (compressible Euler in 1-D, 2-D, 3-D, see below).
 * n_comp:     number of conserved components (1 for the scalar equations,
 *             dim + 2 for Euler: 3, 4 or 5; checked against the mesh).
 * velocity:   advection velocity a (first dim entries used).
 * eps:        epsilon of the non-smoothness indicator, Eq. (smoothness
 *             indicator), e.g. 1e-2; h is the centre cell's mean edge length.
 * alpha_c:    alpha > 1 of the centre weight, Eq. (weight), e.g. 1.5.
 * rank_tol:   numerical rank: #{k : |R_kk| > rank_tol |R_11|}, e.g. 1e-10.
 * kappa_flag: FP32-bulk mode: cells whose conditioning estimate (the spread
 *             max_k/min_k of the column-scaled diagonal |R_kk| / ||R_:,k|| of
 *             the factor of W A) exceeds this get one FP64-residual
 *             refinement sweep (e.g. 1e3); above 1e5 they take the pivoted
 *             path below.
 * precision:  WLSENO_FP64 or WLSENO_FP32_BULK (QR, facet evaluation and the
 *             flux of the deviations in FP32; moments and the refinement
 *             residual in FP64; the reference flux, facet sums, residual and
 *             RK update in FP64 for Euler and in double-float arithmetic --
 *             pairs of FP32 numbers, about 48 bits -- for the scalar
 *             equations, whose FP64 results are hi + lo exactly).
 * gamma:      WLSENO_EULER only: ratio of specific heats (e.g. 1.4).
 * characteristic: WLSENO_EULER only (1-D and 2-D meshes), 0 or 1: reconstruct
 *             characteristic-wise (the characteristic decomposition of
 *             Sec. 5.1.4 and Sec. 5.2.4, per facet on segments and
 *             triangles): for facet f of cell i the stencil
 *             averages are projected onto the eigenvectors of the Jacobian of
 *             F(U).n_f at the mean of the averages of i and its neighbour
 *             across f, each field gets its own weights and least-squares
 *             solve (full-rank stencils, no pivoting), and the traces at f's
 *             points are projected back.  wlseno_reconstruct then returns
 *             facet values only (coeffs must be NULL: there is no single
 *             polynomial per cell); flagged_cells counts (cell, facet) solves
 *             above the flag threshold.
 * balanced:   scalar equations only, 0 or 1: the balanced-stencil
 *             re-selection of Sec. 3.2.  After each reconstruction, a cell
 *             whose value at any of its facet quadrature points leaves
 *             [min, max] of its stencil's averages by more than
 *             balance_margin * (max - min of the averages over its mesh) is
 *             re-solved (FP64) on a stencil of the same size taken from the
 *             (ceil(ring) + 1)-vertex ring: the centre, its facet neighbours
 *             and, on each side of the plane through its centroid normal to
 *             the reconstructed gradient, its nearest cells up to half the
 *             stencil (the side (x_j - x_i).grad u > 0 takes floor(n/2), the
 *             other floor((n-1)/2); a short side is made up from the nearest
 *             remaining cells).  Cells with a zero gradient or an
 *             ill-conditioned new system keep the plain result.  The
 *             re-selected cells are counted in
 *             wlseno_diagnostics.balanced_cells; the adjoint is not available.
 * balance_margin: the range test's margin as a share of the averages' range
 *             (>= 0; e.g. 0.02).
 *
 * WLSENO_EULER (1-D, 2-D, 3-D): n_comp = dim + 2 conserved variables (rho,
 * rho u_1 .. rho u_dim, E), each reconstructed with its own weights
 * (componentwise WLS-ENO; characteristic-wise optional in 1-D and 2-D); LF alpha
 * per facet = max over its points and sides of |u.n| + c; a cell whose traces
 * give density or pressure <= 1e-12 at a facet point uses its averages at all
 * its facets (counted in wlseno_diagnostics.positivity_fallbacks). */
typedef struct {
  int pde;
  int n_comp;
  double velocity[3];
  double eps;
  double alpha_c;
  double rank_tol;
  double kappa_flag;
  int precision;
  double gamma;
  int characteristic;
  int balanced;
  double balance_margin;
} wlseno_scheme;

typedef struct {
  int dim;
  int order_p;
  int m;                   /* Taylor coefficients per cell                      */
  int n_comp;
  int n_meshes;
  int64_t n_cells;         /* over all meshes                                   */
  int64_t stencil_nnz;     /* sum of stencil sizes                              */
  int max_stencil;
  int min_stencil;
  int quad_per_facet;      /* 2 in 2-D, 3 in 3-D                                */
  int lanes_per_cell;      /* kernel shape chosen for the reconstruction        */
  int rows_per_lane;
  int moments_mode;        /* 0 stored rows, 1 formed on the fly (see opts)     */
  int persistent;          /* 1: one persistent kernel per RK step (see opts)   */
} wlseno_info;

/* Kernel kinds of the per-kind launch counts and timings.  RECONSTRUCT is
 * the main reconstruction kernel; FIXUP the follow-ups that redo the cells it
 * flags (refinement sweep, pivoted path) and the balanced-stencil range test
 * and re-selection; DT the per-step preparation (CFL
 * time step and, in FP32-bulk, the FP32 split of the state); STEP the
 * persistent kernel of a whole RK step (opts.persistent). */
enum { WLSENO_KERNEL_MOMENTS = 0, WLSENO_KERNEL_RECONSTRUCT = 1, WLSENO_KERNEL_FLUX = 2,
       WLSENO_KERNEL_DT = 3, WLSENO_KERNEL_ADJOINT = 4, WLSENO_KERNEL_FIXUP = 5,
       WLSENO_KERNEL_STEP = 6, WLSENO_N_KERNEL_KINDS = 7 };

typedef struct {
  int64_t flagged_cells;   /* cells flagged ill-conditioned (last call)         */
  int64_t rank_deficient;  /* cells with numerical rank < m (last call)         */
  int64_t nonfinite;       /* non-finite values seen (last call)                */
  int64_t kernel_launches; /* kernels launched by the context so far            */
  double last_dt;          /* time step of the last rk_step step                */
  int64_t launches_by_kind[WLSENO_N_KERNEL_KINDS]; /* since wlseno_set_timing   */
  double kernel_ms[WLSENO_N_KERNEL_KINDS];         /* summed CUDA-event time of
                                                      each kind since
                                                      wlseno_set_timing (timing
                                                      mode only)                */
  int64_t positivity_fallbacks; /* Euler cells on first order (last call)      */
  int64_t balanced_cells;  /* cells re-solved on balanced stencils, summed over
                              the reconstructions of the last call            */
} wlseno_diagnostics;

/* Create a context on CUDA device `device`; copies *scheme.  When the
 * environment variable WLSENO_DEVICE_BYTES_LIMIT holds a positive decimal
 * integer at this call, the context's device allocations are capped at that
 * many bytes in total: a call whose allocation would pass the cap returns
 * WLSENO_ERR_OOM (as a failed cudaMalloc does) and allocates nothing more
 * (the library's own budget, not the device's free memory).
 * Errors: INVALID_ARG (null, unsupported pde/precision), CUDA. */
wlseno_status wlseno_create(wlseno_ctx** out, int device, const wlseno_scheme* scheme);

/* Release every host and device allocation of the context (NULL is a no-op). */
void wlseno_destroy(wlseno_ctx* ctx);

/* Host setup (Sec. 3.2, Sec. 3.3.1): unwraps cells, computes centroids,
 * volumes, mean edge lengths, facet normals and areas, half-facet siblings
 * and the k-ring stencil of every cell of every mesh (stencils never cross
 * meshes), then uploads them.  The mesh arrays are copied; nothing is kept.
 * perm_out: host [n_cells_total] or NULL; receives for every global cell
 * index of the library's order the caller's global index of that cell
 * (new -> old; the identity unless opts->reorder), so a caller permutes its
 * arrays once: ubar_lib[k] = ubar_caller[perm_out[k]].  Cells never leave
 * their mesh's index range.
 * Errors: INVALID_ARG, MESH (inverted cell, facet shared by > 2 cells),
 * STENCIL (a stencil with fewer than m cells, or more than the kernels hold),
 * OOM, CUDA. */
wlseno_status wlseno_build_stencils(wlseno_ctx* ctx, const wlseno_mesh* meshes, int n_meshes,
                                    const wlseno_stencil_opts* opts, int64_t* perm_out);

/* Device precompute in FP64 (Sec. 3.2, Sec. 3.3.2): for every stencil row
 * (i, j) the h_i-normalised cell average over tau_j of
 * prod_c ((x_c - x_i,c)/h_i)^kappa_c / kappa_c!  (the matrix A of
 * Eq. (average_eq) about the centroid of tau_i), exact by Gauss-Legendre
 * product quadrature on the collapsed simplex; an FP32 copy for FP32-bulk
 * mode; facet quadrature-point offsets.  Must follow wlseno_build_stencils.
 * Errors: STATE, CUDA. */
wlseno_status wlseno_precompute_moments(wlseno_ctx* ctx, void* stream);

/* WLS-ENO reconstruction (Sec. 3.1, Sec. 3.2, Sec. 3.3.2).
 * Solver: each cell's weighted rows are folded into a QR factor of W A
 * without pivoting; when its conditioning estimate stays below the flag
 * threshold (FP32-bulk: kappa_flag; FP64: 1e6) the system has full rank and
 * this is the least-squares solution the paper's pivoted QR returns.  Other
 * cells are redone by Householder QR with column pivoting of W A S, the rank
 * rule of rank_tol and the basic solution (Sec. 3.3.2), or, in FP32-bulk
 * between kappa_flag and 1e5, refined once with the FP64 residual.  With
 * scheme.balanced the cells out of range are then re-solved on balanced
 * stencils (see wlseno_scheme).
 * ubar:   [n_comp][n_cells] cell averages, host or device.
 * coeffs: [n_comp][n_cells][m] output, host or device: h-normalised Taylor
 *         coefficients d_kappa = h_i^|kappa| d^kappa u(x_i) (kappa ordered by
 *         degree, then descending x power), so that
 *         u_i(x) = sum_kappa d_kappa prod_c ((x_c - x_i,c)/h_i)^kappa_c / kappa_c!.
 *         May be NULL.
 * facet_values: [n_comp][n_cells][dim+1][quad_per_facet] output, host or
 *         device, may be NULL: the reconstruction of cell i at the quadrature
 *         points of its local facet f (the facet opposite its local vertex f).
 *         Points are ordered by the facet's vertices sorted by global vertex
 *         index: 1-D the facet's vertex; 2-D Gauss-Legendre t = 1/2 -+ sqrt(3)/6 from the lower to the
 *         higher vertex; 3-D barycentric (2/3,1/6,1/6) on the lowest vertex
 *         first, then the middle, then the highest.
 * Errors: STATE, INVALID_ARG, CUDA, NUMERIC. */
wlseno_status wlseno_reconstruct(wlseno_ctx* ctx, const double* ubar, double* coeffs,
                                 double* facet_values, void* stream);

/* Spatial operator L(ubar) = -(1/|tau_i|) sum over facets of tau_i of the
 * integrated Lax-Friedrichs flux out of tau_i (Sec. 1, Eq. (fvm) divided by
 * |tau_i|, and Eq. (flux)).  Each facet's flux is computed once in the
 * orientation of its lower-indexed cell and used with opposite signs, so the
 * discrete update conserves sum |tau_i| ubar_i to round-off.
 * ubar, residual: [n_comp][n_cells], host or device.
 * Errors: STATE, INVALID_ARG, CUDA, NUMERIC. */
wlseno_status wlseno_flux_residual(wlseno_ctx* ctx, const double* ubar, double* residual,
                                   void* stream);

/* n_steps steps of TVD-RK3 (Sec. 4.2.1, Eq. (3rd-order-Runge-Kutta)) in place.
 * ubar:   [n_comp][n_cells], host or device; overwritten with the result.
 * dt:     > 0: the same fixed step for every mesh;  < 0: the per-mesh fixed
 *         steps given to wlseno_set_mesh_dt;  == 0: each step uses
 *         dt = cfl * min_i r_i / lambda_max with r_i = dim |tau_i| / |d tau_i|
 *         and lambda_max the largest wave speed over the cells (advection |a|,
 *         Burgers sqrt(dim) max |ubar|, Euler max(|u| + c)), computed on the
 *         device per mesh.
 * dt_out: optional host pointer receiving the last step's dt (of mesh 0); it
 *         synchronises the stream when non-NULL.
 * A call with dt > 0 discards the per-mesh steps of wlseno_set_mesh_dt (the
 * fixed step overwrites them on the device): call wlseno_set_mesh_dt again
 * before the next dt < 0 call.
 * One step is captured as a CUDA graph (on the context's own stream) and
 * replayed for n_steps >= 2, for a host ubar (staged through the context's
 * buffer), and for one step whose arguments match the captured one; not in
 * timing mode or while `stream` is being captured.
 * Errors: STATE, INVALID_ARG, CUDA, NUMERIC, TIMEOUT (persistent steps). */
wlseno_status wlseno_rk_step(wlseno_ctx* ctx, double* ubar, double dt, double cfl, int n_steps,
                             double* dt_out, void* stream);

/* The operator of wlseno_flux_residual for callers that cannot allocate
 * device memory when they call it (no paper counterpart: a deployment
 * variant).  Code running inside a stream capture, real-time loops that
 * forbid allocation after start-up and hosts that own all device memory
 * through their own pool cannot call cudaMalloc; this call makes no
 * allocation of any kind.  Its facet-value scratch is a fixed array inside
 * the library (8 MiB of device memory on every GPU that loads the library,
 * held until the process exits), so n_cells * (dim+1) * quad_per_facet may
 * not exceed 1,048,576 (174,762 triangles, 87,381 tetrahedra): larger meshes
 * get WLSENO_ERR_INVALID_ARG and a message.
 * ubar, residual: [n_comp][n_cells] DEVICE arrays (host pointers are rejected
 * with WLSENO_ERR_INVALID_ARG: staging them would allocate).
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  The address is
 * kept for the life of the process: after cudaDeviceReset on that device it
 * is stale, so do not call this entry point again in that process.  Every call shares
 * the one array and fully overwrites the part it reads, so nothing needs
 * clearing, but calls whose work overlaps on the GPU (other streams, other
 * contexts on the same device) race on it: order them on one stream.
 * Errors: STATE, INVALID_ARG, CUDA. */
wlseno_status wlseno_flux_residual_static(wlseno_ctx* ctx, const double* ubar, double* residual,
                                          void* stream);

/* Per-mesh fixed time steps dt_host[n_meshes] (host, all > 0) for
 * wlseno_rk_step and wlseno_step_adjoint called with dt < 0 (a batch of
 * problems each stepping at its own dt).  Errors: STATE, INVALID_ARG, CUDA. */
wlseno_status wlseno_set_mesh_dt(wlseno_ctx* ctx, const double* dt_host);

/* Adjoint of one fixed-dt TVD-RK3 step of wlseno_rk_step (the paper has no
 * adjoint; this differentiates its scheme):
 * gbar_n = (d ubar^{n+1} / d ubar^n)^T gbar_next, including the derivative
 * through the solution-dependent weights omega_j (and the centre's minimum
 * over its facet neighbours) and through the per-facet LF alpha (at its
 * first maximiser); the derivative of the weighted least squares uses its
 * full-rank normal form.  Computed in FP64 kernels with a deterministic
 * transposed-stencil gather (no atomics).
 * ubar_n: the step's input state (checkpoint); the two inner stages are
 * recomputed.  dt: > 0 fixed for every mesh, < 0 the per-mesh steps of
 * wlseno_set_mesh_dt (0 is rejected: a CFL step is not differentiated).
 * All arrays [n_cells] (n_comp = 1), host or device; the first call
 * allocates the adjoint's work arrays.  FP64 contexts, scalar equations on
 * 2-D and 3-D meshes with fixed stencils (balanced = 0), else INVALID_ARG.  A call with
 * dt > 0 discards the steps of wlseno_set_mesh_dt, as in wlseno_rk_step.
 * Errors: STATE, INVALID_ARG, CUDA, NUMERIC. */
wlseno_status wlseno_step_adjoint(wlseno_ctx* ctx, const double* ubar_n, double dt,
                                  const double* gbar_next, double* gbar_n, void* stream);

/* Autotuner: times the reconstruction kernel with every compiled shape
 * (lanes_per_cell, rows_per_lane) whose rows hold the largest stencil (and,
 * for the FP32-bulk thread-per-cell shape, both moments modes), on
 * `ubar` ([n_comp][n_cells], host or device), `reps` launches each after one
 * warm-up launch, and keeps the fastest for the context.  best_us (host,
 * nullable) receives its mean launch time in microseconds.  Synchronises
 * `stream`.  Errors: STATE, INVALID_ARG, CUDA. */
wlseno_status wlseno_autotune(wlseno_ctx* ctx, const double* ubar, int reps, void* stream,
                              double* best_us);

/* Poll limit of the bounded device waits (the grid barriers of the
 * persistent step kernel): a block polls a barrier at most max_polls times,
 * about 64 ns apart, before it gives up; the step then stops at its next
 * barrier in every block, its state is incomplete, and the next call on the
 * context (or this rk_step call, when it synchronises) returns
 * WLSENO_ERR_TIMEOUT.  0 restores the default 2^24 (about a second).
 * Host only; takes effect at the next step that is not a replay of an
 * already captured one (the limit is part of the captured launch).
 * Errors: INVALID_ARG (null context, max_polls < 0). */
wlseno_status wlseno_set_wait_limit(wlseno_ctx* ctx, int64_t max_polls);

/* Sizes and the kernel shape in use.  Errors: STATE, INVALID_ARG. */
wlseno_status wlseno_get_info(const wlseno_ctx* ctx, wlseno_info* out);

/* Host copies of the stencils: row_ptr [n_cells+1], cols [stencil_nnz]
 * (global cell indices, centre cell first, then increasing index).
 * Errors: STATE, INVALID_ARG. */
wlseno_status wlseno_get_stencils(const wlseno_ctx* ctx, int64_t* row_ptr, int64_t* cols);

/* Host copies of per-cell geometry (any pointer may be NULL):
 * centroid [n_cells][dim], volume [n_cells], h [n_cells] (mean edge length),
 * inradius [n_cells].  Errors: STATE. */
wlseno_status wlseno_get_geometry(const wlseno_ctx* ctx, double* centroid, double* volume,
                                  double* h, double* inradius);

/* Counters of the last call (synchronises the context's last stream). */
wlseno_status wlseno_get_diagnostics(wlseno_ctx* ctx, wlseno_diagnostics* out);

/* Timing mode: enable != 0 records a CUDA event pair on the launching stream
 * around every kernel the context launches; wlseno_get_diagnostics sums them
 * per kernel kind.  Each wlseno_set_timing call resets the per-kind counts
 * and times; otherwise they accumulate over calls.
 * Errors: INVALID_ARG, CUDA. */
wlseno_status wlseno_set_timing(wlseno_ctx* ctx, int enable);

/* Measured arithmetic peak of device `device` for the rooflines of a
 * benchmark (no counterpart in the paper: a measurement utility).
 * precision WLSENO_FP32_BULK measures FP32, WLSENO_FP64 FP64 fused
 * multiply-add throughput: independent FMA chains (8 per thread, 256 threads
 * per block, 8 blocks per SM), the fastest of five timed launches after one
 * warm-up, 2 flops per FMA, in TFLOP/s into *tflops (host).  Runs on the
 * legacy default stream and synchronises; allocates a small device buffer;
 * reads and changes no GPU setting.  Errors: INVALID_ARG, CUDA, OOM. */
wlseno_status wlseno_measure_fma_peak(int device, int precision, double* tflops);

const char* wlseno_status_string(wlseno_status s);

/* Human-readable detail of the last error the context reported ("" if none). */
const char* wlseno_last_error_message(const wlseno_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* WLSENO_H */
