// Test probe for the CPU suite: the library's Hilbert cell order
// (csrc/reorder.cpp) compiled as host C++.  Reads "dim nv nc", the nv
// vertices (dim coordinates each), the nc cells (dim+1 indices each) and the
// dim periods; prints the new -> old order, one index per line.
#include <cstdio>
#include <vector>

#include "wlseno_internal.h"

int main() {
  int dim = 0;
  long long nv = 0, nc = 0;
  if (std::scanf("%d %lld %lld", &dim, &nv, &nc) != 3) return 2;
  std::vector<double> v(nv * dim), period(dim);
  std::vector<int64_t> cells(nc * (dim + 1));
  for (auto& x : v)
    if (std::scanf("%lf", &x) != 1) return 2;
  for (auto& c : cells) {
    long long t = 0;
    if (std::scanf("%lld", &t) != 1) return 2;
    c = t;
  }
  for (auto& p : period)
    if (std::scanf("%lf", &p) != 1) return 2;
  wlseno_mesh m{dim, nv, nc, v.data(), cells.data(), period.data()};
  std::vector<int64_t> order;
  if (!wlseno::hilbert_order(m, &order)) return 3;
  for (int64_t k : order) std::printf("%lld\n", static_cast<long long>(k));
  return 0;
}
