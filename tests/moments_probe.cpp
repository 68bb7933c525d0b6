// Test probe for the CPU suite: the library's FP64 moment rows
// (csrc/moment_row.cuh, the quadrature the device precompute and the
// balanced re-selection use) evaluated on the host, on the stencils of the
// native host setup, for a mesh read from stdin (the format of
// host_setup_probe.cpp).  Prints "rows <count> ..." with the m entries of
// every stencil row, cell by cell in stencil order.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>
#include <vector>

#include "moment_row.cuh"
#include "wlseno_internal.h"

namespace {

template <int DIM, int M>
void rows(const wlseno::HostSetup& H, const wlseno::DeviceMesh& dm) {
  const wlseno::GaussRule g = wlseno::make_gauss_rule();
  std::printf("rows %lld", static_cast<long long>(H.nnz * M));
  for (int64_t i = 0; i < H.N; ++i)
    for (int64_t e = H.row_ptr[i]; e < H.row_ptr[i + 1]; ++e) {
      double acc[M];
      wlseno::moment_row<DIM, M>(dm, g, i, H.cols[e], acc);
      for (int c = 0; c < M; ++c) std::printf(" %.17g", acc[c]);
    }
  std::printf("\n");
}

}  // namespace

int main() {
  int dim = 0, order_p = 0, min_rows = 0, balance_steps = 0;
  long long nv = 0, nc = 0;
  double ring = 0.0, radius_cut = 0.0;
  if (std::scanf("%d %lld %lld %d %lf %lf %d %d", &dim, &nv, &nc, &order_p, &ring, &radius_cut, &min_rows,
                 &balance_steps) != 8)
    return 2;
  std::vector<double> period(dim), vertices(static_cast<size_t>(nv) * dim);
  std::vector<int64_t> cells(static_cast<size_t>(nc) * (dim + 1));
  for (auto& x : period)
    if (std::scanf("%lf", &x) != 1) return 2;
  for (auto& x : vertices)
    if (std::scanf("%lf", &x) != 1) return 2;
  for (auto& c : cells) {
    long long v = 0;
    if (std::scanf("%lld", &v) != 1) return 2;
    c = v;
  }
  wlseno_mesh mesh{dim, nv, nc, vertices.data(), cells.data(), period.data()};
  wlseno_stencil_opts opts{};
  opts.order_p = order_p;
  opts.ring = ring;
  opts.radius_cut = radius_cut;
  opts.min_rows = min_rows;
  wlseno::HostSetup H;
  std::string err;
  if (wlseno::build_host_setup(&mesh, 1, &opts, &H, &err) != WLSENO_OK) {
    std::printf("error %s\n", err.c_str());
    return 1;
  }
  wlseno::DeviceMesh dm{};
  dm.dim = H.dim;
  dm.m = H.m;
  dm.N = H.N;
  dm.coords = H.coords.data();
  dm.centroid = H.centroid.data();
  dm.h = H.h.data();
  dm.mesh_of = H.mesh_of.data();
  dm.period = H.period.data();
  if (dim == 1 && H.m == 3) rows<1, 3>(H, dm);
  else if (dim == 1 && H.m == 5) rows<1, 5>(H, dm);
  else if (dim == 2 && H.m == 6) rows<2, 6>(H, dm);
  else if (dim == 2 && H.m == 10) rows<2, 10>(H, dm);
  else if (dim == 3 && H.m == 10) rows<3, 10>(H, dm);
  else return 3;
  return 0;
}
