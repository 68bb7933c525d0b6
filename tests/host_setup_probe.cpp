// Test probe for the CPU suite: runs the library's native host setup
// (build_host_setup: geometry, facet records, k-ring stencils and the
// balanced-stencil candidates) on one mesh read from stdin and prints its
// results, so that the host logic is checked against the oracle without a
// GPU.  Built by tests/test_host_setup.py together with csrc/host_mesh.cpp.
//
// stdin (whitespace separated): dim n_vertices n_cells order_p ring
// radius_cut min_rows balance_steps, period[dim], vertices[n_vertices][dim],
// cells[n_cells][dim+1].
// stdout: "status <code> <message>", then one line per array:
// "<name> <count> v0 v1 ...".
#include <cstdio>
#include <string>
#include <type_traits>
#include <vector>

#include "wlseno_internal.h"

namespace {

template <typename T>
void print_array(const char* name, const std::vector<T>& v) {
  std::printf("%s %zu", name, v.size());
  for (const T& x : v) {
    if constexpr (std::is_floating_point<T>::value)
      std::printf(" %.17g", static_cast<double>(x));
    else
      std::printf(" %lld", static_cast<long long>(x));
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
  const wlseno_status st = wlseno::build_host_setup(&mesh, 1, &opts, &H, &err, balance_steps);
  std::printf("status %d %s\n", static_cast<int>(st), err.empty() ? "-" : err.c_str());
  if (st != WLSENO_OK) return 0;
  print_array("row_ptr", H.row_ptr);
  print_array("cols", H.cols);
  print_array("centroid", H.centroid);
  print_array("volume", H.volume);
  print_array("h", H.h);
  print_array("inradius", H.inradius);
  print_array("nbr", H.nbr);
  print_array("fgeo", H.fgeo);
  print_array("bal_ptr", H.bal_ptr);
  print_array("bal_idx", H.bal_idx);
  return 0;
}
