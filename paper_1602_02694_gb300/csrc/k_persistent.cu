// One TVD-RK3 step (Sec. 4.2.1) of the scalar equations as ONE persistent
// cooperative kernel: every block stays resident for the whole step and walks
// the cells of all meshes of the context (a batch of meshes of uneven sizes
// is one concatenated cell range, the cells of a mesh contiguous) through
//   the wave-speed pass (CFL time step per mesh) and the state's FP32 pairs,
//   then per stage: the thread-per-cell reconstruction, the follow-ups on the
//   cells it flagged (FP64-residual refinement, pivoted path), and the
//   Lax-Friedrichs flux with the Shu-Osher combination,
// separated by grid-wide barriers.  The phases run the same per-cell bodies
// as the kernel-per-phase step (k_recon_tpc_kernels.cuh, k_reconstruct.cuh,
// k_flux_cell.cuh), so both give the same bits.
//
// Every barrier wait is bounded: a block polls the barrier's generation at
// most spin_cap times (about 64 ns apart); past that it sets the launch's
// status word, raises the context's host-visible timeout word (the next
// entry point returns WLSENO_ERR_TIMEOUT) and returns, and every other block
// gives up at its next barrier.  No wait is unbounded and nothing traps.
//
// Arrays written by one phase are read by later phases of the same launch,
// so the bodies are compiled here without __restrict__ (no non-coherent
// loads); the barrier's acquire/release pair orders those writes and reads.
#define WLSENO_BODY_RESTRICT
#include "k_flux_cell.cuh"
#include "k_recon_tpc_kernels.cuh"
#include "k_reconstruct.cuh"

namespace wlseno {
namespace {

struct PersistArgs {
  DeviceMesh dm;
  SchemeParams sp;
  double* u;
  double* k1;
  double* k2;
  float2* pu;  // FP32 pairs of u, k1, k2 (FP32-bulk)
  float2* p1;
  float2* p2;
  double* fvals;  // FP64 facet values, or the FP32 deviations fdev in FP32-bulk
  float* fdev;
  unsigned long long* counters;
  int* group_list;
  int* counts;  // [3][2] per stage: pivoted-list and refine-record lengths (zero at launch)
  float* refine_buf;
  int64_t capacity;
  int dt_mode;  // 0: CFL step from the state; 1: dt_fixed; 2: the per-mesh steps already in dt_mesh
  double cfl, dt_fixed;
  double adv_speed;  // advection |a| (the CFL step's wave speed)
  float speed;       // the same in FP32 (the FP32-bulk flux)
  int n_meshes;
  const double* rmin;
  unsigned long long* lmax;  // [n_meshes] (zero at launch)
  double* dt_mesh;
  float2* dt2;
  unsigned int* bar;     // [2] arrivals, generation (zero at launch)
  int* status;           // 1 once a wait gave up (zero at launch)
  unsigned int* timeout_word;  // the context's host-visible timeout word
  long long spin_cap;
  double flag, pivot;    // thresholds of the reconstruction (as launch_recon_tpc)
};

// Grid-wide barrier with a bounded wait.  Returns false when this or another
// block gave up (the caller returns).
__device__ __forceinline__ bool grid_sync(const PersistArgs& a) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int gen, prev;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(a.bar + 1) : "memory");
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(a.bar) : "memory");
    if (prev == gridDim.x - 1) {
      // last arrival: reset the count for the next barrier, then release
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a.bar), "r"(0u) : "memory");
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a.bar + 1), "r"(gen + 1u) : "memory");
    } else {
      long long spins = 0;
      while (true) {
        unsigned int g;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(a.bar + 1) : "memory");
        if (g != gen) break;
        if (*reinterpret_cast<volatile int*>(a.status) != 0) {
          ok = 0;
          break;
        }
        if (++spins > a.spin_cap) {
          atomicExch(a.status, 1);
          *reinterpret_cast<volatile unsigned int*>(a.timeout_word) = 1u;
          __threadfence_system();
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    if (*reinterpret_cast<volatile int*>(a.status) != 0) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T, int DIM, int M, bool OTF, int LG, int LR>
__global__ void __launch_bounds__(128, 2) persistent_step_kernel(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool F32 = sizeof(T) == 4;
  const int64_t N = a.dm.N;
  const int64_t nthr = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t gt0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  // wave speeds per mesh (Burgers CFL steps) and the FP32 pairs of u
  if (a.dt_mode == 0 && a.sp.pde == WLSENO_BURGERS) {
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < N; base += nthr) {
      const int64_t i = base + threadIdx.x;  // whole warps take part (warp reduction)
      max_abs_cell(N, a.u, a.dm.mesh_of, a.lmax, F32 ? a.pu : nullptr, i, i < N);
    }
  } else if (F32) {
    for (int64_t i = gt0; i < N; i += nthr) {
      const dfloat d = df_from_double_bits(a.u[i]);
      a.pu[i] = make_float2(d.hi, d.lo);
    }
  }
  if (!grid_sync(a)) return;
  if (blockIdx.x == 0 && a.dt_mode != 2) {
    // the time step of every mesh (read by the first flux phase, two
    // barriers later)
    for (int k = threadIdx.x; k < a.n_meshes; k += blockDim.x) {
      // (the maxima exist for CFL steps of Burgers only: advection has |a|)
      const unsigned long long bits = a.lmax ? reinterpret_cast<volatile unsigned long long*>(a.lmax)[k] : 0ull;
      const double dt = cfl_dt_of(a.sp.pde, DIM, a.adv_speed, bits, a.rmin[k], a.cfl,
                                  a.dt_mode == 1 ? a.dt_fixed : 0.0);
      a.dt_mesh[k] = dt;
      if (a.dt2) {
        const dfloat v = df_from_double(dt);
        a.dt2[k] = make_float2(v.hi, v.lo);
      }
    }
  }
  // k1 = u + dt L(u);  k2 = 3/4 u + 1/4 (k1 + dt L(k1));  u <- 1/3 u + 2/3 (k2 + dt L(k2))
  double* xin[3] = {a.u, a.k1, a.k2};
  double* xout[3] = {a.k1, a.k2, a.u};
  float2* pin[3] = {a.pu, a.p1, a.p2};
  float2* pout[3] = {a.p1, a.p2, nullptr};
  const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
  const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
  const T flag = static_cast<T>(a.flag), pivot = static_cast<T>(a.pivot);
  double* fv = F32 ? nullptr : a.fvals;
  float* fd = F32 ? a.fdev : nullptr;
#pragma unroll 1
  for (int s = 0; s < 3; ++s) {
    TpcWork w{a.group_list, a.counts + 2 * s, F32 ? a.refine_buf : nullptr, F32 ? pin[s] : nullptr,
              nullptr, nullptr, nullptr, OTF};
    w.capacity = a.capacity;
    for (int64_t gt = gt0; gt < N; gt += nthr)
      recon_tpc_cell<T, DIM, M, OTF, 1>(a.dm, a.sp, xin[s], nullptr, fv, fd, a.counters, w, flag, pivot, gt);
    if (!grid_sync(a)) return;
    if constexpr (F32) refine_records<DIM, M, 16, 4>(a.dm, xin[s], nullptr, fv, fd, w, gt0, nthr);
    reconstruct_listed<T, DIM, M, LG, LR>(a.dm, a.sp, xin[s], nullptr, fv, fd, a.counters, a.group_list, w.counts,
                                          smem_raw, blockIdx.x, gridDim.x);
    if (!grid_sync(a)) return;
    for (int64_t i = gt0; i < N; i += nthr) {
      if constexpr (F32)
        flux_df_cell<DIM>(a.dm, a.sp.pde, a.speed, a.fdev, pin[s], a.pu, df_from_double(ca[s]),
                          df_from_double(cb[s]), a.dt2, 0, xout[s], a.counters, pout[s], i);
      else
        flux_cell<double, DIM>(a.dm, a.sp, a.fvals, xin[s], a.u, ca[s], cb[s], a.dt_mesh, 0, xout[s], a.counters,
                               i);
    }
    if (s < 2 && !grid_sync(a)) return;
  }
}

template <typename T, int DIM, int M, bool OTF, int LG, int LR>
cudaError_t launch_shape(const PersistArgs& a, cudaStream_t s) {
  auto fn = persistent_step_kernel<T, DIM, M, OTF, LG, LR>;
  constexpr int threads = 128;
  const size_t smem = recon_smem_per_cell<T, M, LG, LR>() * (threads / LG);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int64_t need = (a.dm.N + threads - 1) / threads;
  const int64_t cap = static_cast<int64_t>(per_sm) * sms;
  const unsigned blocks = static_cast<unsigned>(need < cap ? (need > 0 ? need : 1) : cap);
  PersistArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(fn), dim3(blocks), dim3(threads), params, smem,
                                     s);
}

}  // namespace

bool persistent_supported(int dim, int m) { return dim == 2 && (m == 6 || m == 10); }

cudaError_t launch_persistent_step(const PersistLaunch& L, cudaStream_t s) {
  const DeviceMesh& dm = L.dm;
  if (!persistent_supported(dm.dim, dm.m) || dm.nmax > 64) return cudaErrorInvalidValue;
  PersistArgs a{};
  a.dm = dm;
  a.sp = L.sp;
  a.u = L.u;
  a.k1 = L.k1;
  a.k2 = L.k2;
  a.pu = L.pairs;
  a.p1 = L.pairs ? L.pairs + dm.N : nullptr;
  a.p2 = L.pairs ? L.pairs + 2 * dm.N : nullptr;
  a.fvals = L.fvals;
  a.fdev = L.fdev;
  a.counters = L.counters;
  a.group_list = L.group_list;
  a.counts = L.counts;
  a.refine_buf = L.refine_buf;
  a.capacity = L.capacity;
  a.dt_mode = L.dt_mode;
  a.cfl = L.cfl;
  a.dt_fixed = L.dt_fixed;
  a.speed = static_cast<float>(L.adv_speed);
  a.adv_speed = L.adv_speed;
  a.n_meshes = L.n_meshes;
  a.rmin = L.rmin;
  a.lmax = L.lmax;
  a.dt_mesh = L.dt_mesh;
  a.dt2 = L.dt2;
  a.bar = L.sync_words;
  a.status = reinterpret_cast<int*>(L.sync_words + 2);
  a.timeout_word = L.timeout_word;
  a.spin_cap = L.spin_cap;
  a.flag = L.flag;
  a.pivot = L.pivot;
  // zeroed launch state: per-stage list lengths, wave-speed maxima, barrier
  cudaError_t e = cudaMemsetAsync(L.counts, 0, 6 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.sync_words, 0, 3 * sizeof(unsigned int), s);
  if (e == cudaSuccess && L.lmax) e = cudaMemsetAsync(L.lmax, 0, sizeof(unsigned long long) * L.n_meshes, s);
  if (e != cudaSuccess) return e;
  const bool big = dm.nmax > 40;  // list shape: (8 lanes x 5 rows) or (16 x 4)
  if (L.fp32) {
    if (!L.pairs || !L.fdev || !L.refine_buf || !L.dt2) return cudaErrorInvalidValue;
    if (dm.m == 6)
      return L.otf ? (big ? launch_shape<float, 2, 6, true, 16, 4>(a, s) : launch_shape<float, 2, 6, true, 8, 5>(a, s))
                   : (big ? launch_shape<float, 2, 6, false, 16, 4>(a, s) : launch_shape<float, 2, 6, false, 8, 5>(a, s));
    return L.otf ? (big ? launch_shape<float, 2, 10, true, 16, 4>(a, s) : launch_shape<float, 2, 10, true, 8, 5>(a, s))
                 : (big ? launch_shape<float, 2, 10, false, 16, 4>(a, s) : launch_shape<float, 2, 10, false, 8, 5>(a, s));
  }
  if (!L.fvals) return cudaErrorInvalidValue;
  if (dm.m == 6)
    return big ? launch_shape<double, 2, 6, false, 16, 4>(a, s) : launch_shape<double, 2, 6, false, 8, 5>(a, s);
  return big ? launch_shape<double, 2, 10, false, 16, 4>(a, s) : launch_shape<double, 2, 10, false, 8, 5>(a, s);
}

}  // namespace wlseno
