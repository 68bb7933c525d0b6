// Cell reordering for locality (host, native C++): each mesh's cells sorted
// by the Hilbert index of their centroids, so that stencil neighbours sit at
// nearby indices and the gathers of the reconstruction and flux kernels touch
// few distinct cache lines whatever order the caller's mesh came in.
//
// The Hilbert index is computed by Skilling's transform ("Programming the
// Hilbert curve", AIP Conf. Proc. 707, 2004): the integer coordinates of a
// point, b bits each, are turned in place into the "transposed" Hilbert
// index (an inverse-undo pass over the bit planes, then Gray encoding), whose
// bits interleaved from the top plane down form the index.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "wlseno_internal.h"

namespace wlseno {
namespace {

// In place: coordinates x[0..n) of b bits -> transposed Hilbert index.
void axes_to_transpose(uint32_t* x, int b, int n) {
  const uint32_t top = 1u << (b - 1);
  for (uint32_t q = top; q > 1; q >>= 1) {
    const uint32_t p = q - 1;
    for (int i = 0; i < n; ++i) {
      if (x[i] & q) {
        x[0] ^= p;  // invert the low bits of x[0]
      } else {      // exchange the low bits of x[0] and x[i]
        const uint32_t t = (x[0] ^ x[i]) & p;
        x[0] ^= t;
        x[i] ^= t;
      }
    }
  }
  for (int i = 1; i < n; ++i) x[i] ^= x[i - 1];  // Gray encode
  uint32_t t = 0;
  for (uint32_t q = top; q > 1; q >>= 1)
    if (x[n - 1] & q) t ^= q - 1;
  for (int i = 0; i < n; ++i) x[i] ^= t;
}

uint64_t hilbert_key(const double* c, const double* lo, const double* span, int n) {
  const int b = n == 1 ? 32 : n == 2 ? 31 : 21;
  const double cells = std::ldexp(1.0, b);
  uint32_t x[3] = {0, 0, 0};
  for (int a = 0; a < n; ++a) {
    double v = span[a] > 0.0 ? (c[a] - lo[a]) / span[a] * cells : 0.0;
    v = std::min(std::max(v, 0.0), cells - 1.0);
    x[a] = static_cast<uint32_t>(v);
  }
  if (n == 1) return x[0];
  axes_to_transpose(x, b, n);
  uint64_t key = 0;
  for (int bit = b - 1; bit >= 0; --bit)
    for (int a = 0; a < n; ++a) key = (key << 1) | ((x[a] >> bit) & 1u);
  return key;
}

}  // namespace

// new_to_old[k] for the cells of one mesh (local indices): sorted by the
// Hilbert key of the centroid (periodic axes: each cell's vertices taken at
// their minimum image about its first vertex, the centroid wrapped into the
// period), ties by the original index.  Returns false on a bad cell index.
bool hilbert_order(const wlseno_mesh& m, std::vector<int64_t>* new_to_old) {
  const int d = m.dim, nv = d + 1;
  std::vector<double> cen(static_cast<size_t>(m.n_cells) * d);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cell = m.cells + c * nv;
    for (int k = 0; k < nv; ++k)
      if (cell[k] < 0 || cell[k] >= m.n_vertices) return false;
    for (int a = 0; a < d; ++a) {
      const double x0 = m.vertices[cell[0] * d + a];
      const double per = m.period ? m.period[a] : 0.0;
      double s = 0.0;
      for (int k = 0; k < nv; ++k) {
        double dx = m.vertices[cell[k] * d + a] - x0;
        if (per > 0.0) dx -= per * std::round(dx / per);
        s += dx;
      }
      double v = x0 + s / nv;
      if (per > 0.0) v -= per * std::floor(v / per);
      cen[c * d + a] = v;
    }
  }
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, span[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    lo[a] = INFINITY;
    hi[a] = -INFINITY;
    for (int64_t c = 0; c < m.n_cells; ++c) {
      lo[a] = std::min(lo[a], cen[c * d + a]);
      hi[a] = std::max(hi[a], cen[c * d + a]);
    }
    span[a] = hi[a] - lo[a];
  }
  // one scale for every axis keeps the curve's cells square
  const double s = *std::max_element(span, span + d);
  for (int a = 0; a < d; ++a) span[a] = s;
  std::vector<uint64_t> key(m.n_cells);
  for (int64_t c = 0; c < m.n_cells; ++c) key[c] = hilbert_key(&cen[c * d], lo, span, d);
  new_to_old->resize(m.n_cells);
  std::iota(new_to_old->begin(), new_to_old->end(), int64_t(0));
  std::stable_sort(new_to_old->begin(), new_to_old->end(),
                   [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  return true;
}

}  // namespace wlseno
