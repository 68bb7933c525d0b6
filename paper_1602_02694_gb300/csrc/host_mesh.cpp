// Host setup of libwlseno: cell geometry, half-facet siblings (Sec. 3.3.1),
// k-ring stencils with 1/2- and 1/3-ring increments (Sec. 3.2) and the facet
// data the flux kernel streams (owner-oriented normals, areas, quadrature
// points).  Plain C++, O(N * stencil) time.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "wlseno_internal.h"

namespace wlseno {
namespace {

inline double wrap_delta(double d, double L) { return L > 0.0 ? d - L * std::nearbyint(d / L) : d; }

int n_coeffs(int dim, int p) {
  // C(p-1+dim, dim)
  int num = 1, den = 1;
  for (int k = 1; k <= dim; ++k) {
    num *= (p - 1 + k);
    den *= k;
  }
  return num / den;
}

double det3(const double* a, const double* b, const double* c) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
         a[2] * (b[0] * c[1] - b[1] * c[0]);
}

// Ring increments of Sec. 3.2 as a list of step kinds.
enum Step { kFacet = 0, kEdge = 1, kVertex = 2 };

bool ring_steps(int dim, double ring, std::vector<int>* steps) {
  steps->clear();
  if (!(ring > 0.0) || ring > 8.0) return false;
  int whole = static_cast<int>(std::floor(ring + 1e-9));
  double frac = ring - whole;
  for (int k = 0; k < whole; ++k) steps->push_back(kVertex);
  if (std::fabs(frac) < 1e-6) return !steps->empty();
  if (dim == 2 && std::fabs(frac - 0.5) < 1e-6) {
    steps->push_back(kFacet);
    return true;
  }
  if (dim == 3 && std::fabs(frac - 1.0 / 3.0) < 1e-3) {
    steps->push_back(kFacet);
    return true;
  }
  if (dim == 3 && std::fabs(frac - 2.0 / 3.0) < 1e-3) {
    steps->push_back(kEdge);
    return true;
  }
  return false;
}

struct MeshWork {
  int dim = 0;
  int64_t nc = 0, nv = 0;
  const int64_t* cells = nullptr;
  std::vector<int64_t> inc_ptr, inc;    // vertex -> incident cells (CSR)
  std::vector<int64_t> sib;             // [nc][dim+1]: sibling cell or -1
  std::vector<int8_t> sib_f;            // [nc][dim+1]: sibling local facet
};

// Cells incident to both vertices a and b (sorted incidence lists).
template <typename F>
void for_cells_sharing_edge(const MeshWork& w, int64_t a, int64_t b, F&& fn) {
  const int64_t* pa = w.inc.data() + w.inc_ptr[a];
  const int64_t* ea = w.inc.data() + w.inc_ptr[a + 1];
  const int64_t* pb = w.inc.data() + w.inc_ptr[b];
  const int64_t* eb = w.inc.data() + w.inc_ptr[b + 1];
  while (pa < ea && pb < eb) {
    if (*pa < *pb) ++pa;
    else if (*pb < *pa) ++pb;
    else {
      fn(*pa);
      ++pa;
      ++pb;
    }
  }
}

}  // namespace

wlseno_status build_host_setup(const wlseno_mesh* meshes, int n_meshes,
                               const wlseno_stencil_opts* opts, HostSetup* out,
                               std::string* err, int balance_steps) {
  if (!meshes || n_meshes <= 0 || !opts || !out) {
    *err = "null argument or n_meshes <= 0";
    return WLSENO_ERR_INVALID_ARG;
  }
  const int dim = meshes[0].dim;
  if (dim < 1 || dim > 3) {
    *err = "dim must be 1, 2 or 3";
    return WLSENO_ERR_INVALID_ARG;
  }
  const int p = opts->order_p;
  if ((dim == 1 && p != 3 && p != 5) || (dim == 2 && (p < 3 || p > 4)) || (dim == 3 && p != 3)) {
    *err = "unsupported order p for this dimension";
    return WLSENO_ERR_INVALID_ARG;
  }
  std::vector<int> steps;
  if (!ring_steps(dim, opts->ring, &steps)) {
    *err = "ring is not a positive integer (1-D) or multiple of 1/2 (2-D) or 1/3 (3-D)";
    return WLSENO_ERR_INVALID_ARG;
  }
  const int m = n_coeffs(dim, p);
  const int min_rows = opts->min_rows > 0 ? opts->min_rows : (3 * m + 1) / 2;
  const int nf = dim + 1;
  const int nq = nq_of(dim);

  HostSetup& S = *out;
  S = HostSetup();
  S.dim = dim;
  S.p = p;
  S.m = m;
  S.nq = nq;
  S.n_meshes = n_meshes;
  int64_t N = 0;
  for (int k = 0; k < n_meshes; ++k) {
    const wlseno_mesh& M = meshes[k];
    if (M.dim != dim || M.n_cells <= 0 || M.n_vertices <= 0 || !M.vertices || !M.cells ||
        !M.period) {
      *err = "mesh " + std::to_string(k) + ": bad dim, sizes or null arrays";
      return WLSENO_ERR_INVALID_ARG;
    }
    N += M.n_cells;
  }
  if (N >= (int64_t(1) << 29)) {
    *err = "too many cells for 32-bit stencil indices";
    return WLSENO_ERR_INVALID_ARG;
  }
  S.N = N;
  S.coords.assign(N * nf * dim, 0.0);
  S.centroid.assign(N * dim, 0.0);
  S.volume.assign(N, 0.0);
  S.h.assign(N, 0.0);
  S.inradius.assign(N, 0.0);
  S.mesh_of.assign(N, 0);
  S.period.assign(n_meshes * 3, 0.0);
  S.rmin.assign(n_meshes, 0.0);
  S.nbr.assign(N * nf, -1);
  S.fgeo.assign(N * nf * 4, 0.0);
  S.fpts.assign(N * nf * nq * dim, 0.0);
  S.row_ptr.assign(N + 1, 0);
  if (balance_steps > 0) S.bal_ptr.assign(N + 1, 0);
  S.cols.clear();

  std::vector<double> own_normal(N * nf * 3, 0.0), own_area(N * nf, 0.0);
  int64_t base = 0;
  for (int k = 0; k < n_meshes; ++k) {
    const wlseno_mesh& M = meshes[k];
    const int64_t nc = M.n_cells, nv = M.n_vertices;
    double L[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      L[a] = M.period[a];
      S.period[k * 3 + a] = L[a];
      if (!(L[a] >= 0.0)) {
        *err = "negative period";
        return WLSENO_ERR_INVALID_ARG;
      }
    }
    // ---- geometry of every cell, unwrapped relative to its first vertex
    double rmin = 1e300;
    for (int64_t c = 0; c < nc; ++c) {
      const int64_t gc = base + c;
      S.mesh_of[gc] = k;
      double* X = &S.coords[gc * nf * dim];
      for (int v = 0; v < nf; ++v) {
        int64_t vid = M.cells[c * nf + v];
        if (vid < 0 || vid >= nv) {
          *err = "mesh " + std::to_string(k) + ": vertex index out of range in cell " +
                 std::to_string(c);
          return WLSENO_ERR_MESH;
        }
        for (int a = 0; a < dim; ++a) {
          double x0 = M.vertices[M.cells[c * nf] * dim + a];
          X[v * dim + a] = x0 + wrap_delta(M.vertices[vid * dim + a] - x0, L[a]);
        }
      }
      double e[3][3];
      for (int v = 1; v < nf; ++v)
        for (int a = 0; a < dim; ++a) e[v - 1][a] = X[v * dim + a] - X[a];
      double vol = dim == 1   ? e[0][0]
                   : dim == 2 ? 0.5 * (e[0][0] * e[1][1] - e[0][1] * e[1][0])
                              : det3(e[0], e[1], e[2]) / 6.0;
      if (!(vol > 0.0)) {
        *err = "mesh " + std::to_string(k) + ": cell " + std::to_string(c) +
               " is inverted or degenerate";
        return WLSENO_ERR_MESH;
      }
      S.volume[gc] = vol;
      double edge_sum = 0.0;
      int n_edges = 0;
      for (int a = 0; a < nf; ++a)
        for (int b = a + 1; b < nf; ++b) {
          double s2 = 0.0;
          for (int q = 0; q < dim; ++q) {
            double d = X[b * dim + q] - X[a * dim + q];
            s2 += d * d;
          }
          edge_sum += std::sqrt(s2);
          ++n_edges;
        }
      S.h[gc] = edge_sum / n_edges;
      for (int a = 0; a < dim; ++a) {
        double s = 0.0;
        for (int v = 0; v < nf; ++v) s += X[v * dim + a];
        S.centroid[gc * dim + a] = s / nf;
      }
      // outward normals and areas of the facets (facet f is opposite vertex f)
      double bnd = 0.0;
      for (int f = 0; f < nf; ++f) {
        int loc[3], t = 0;
        for (int v = 0; v < nf; ++v)
          if (v != f) loc[t++] = v;
        double n[3] = {0, 0, 0}, area;
        if (dim == 1) {  // the facet is the vertex loc[0]: unit measure
          area = 1.0;
          n[0] = 1.0;
        } else if (dim == 2) {
          double ex = X[loc[1] * 2] - X[loc[0] * 2], ey = X[loc[1] * 2 + 1] - X[loc[0] * 2 + 1];
          area = std::sqrt(ex * ex + ey * ey);
          n[0] = ey / area;
          n[1] = -ex / area;
        } else {
          double u[3], w[3];
          for (int a = 0; a < 3; ++a) {
            u[a] = X[loc[1] * 3 + a] - X[loc[0] * 3 + a];
            w[a] = X[loc[2] * 3 + a] - X[loc[0] * 3 + a];
          }
          double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2],
                 cz = u[0] * w[1] - u[1] * w[0];
          double len = std::sqrt(cx * cx + cy * cy + cz * cz);
          area = 0.5 * len;
          n[0] = cx / len;
          n[1] = cy / len;
          n[2] = cz / len;
        }
        // orient away from the opposite vertex
        double dot = 0.0;
        for (int a = 0; a < dim; ++a) dot += (X[loc[0] * dim + a] - X[f * dim + a]) * n[a];
        if (dot < 0.0)
          for (int a = 0; a < dim; ++a) n[a] = -n[a];
        for (int a = 0; a < dim; ++a) own_normal[(gc * nf + f) * 3 + a] = n[a];
        own_area[gc * nf + f] = area;
        bnd += area;
      }
      S.inradius[gc] = dim * vol / bnd;
      rmin = std::min(rmin, S.inradius[gc]);
    }
    S.rmin[k] = rmin;

    // ---- vertex -> cell incidence
    MeshWork w;
    w.dim = dim;
    w.nc = nc;
    w.nv = nv;
    w.cells = M.cells;
    w.inc_ptr.assign(nv + 1, 0);
    for (int64_t i = 0; i < nc * nf; ++i) w.inc_ptr[M.cells[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) w.inc_ptr[v + 1] += w.inc_ptr[v];
    w.inc.assign(nc * nf, 0);
    {
      std::vector<int64_t> fill(w.inc_ptr.begin(), w.inc_ptr.end() - 1);
      for (int64_t c = 0; c < nc; ++c)
        for (int v = 0; v < nf; ++v) w.inc[fill[M.cells[c * nf + v]]++] = c;  // ascending c
    }
    // ---- half-facet siblings: sort facet keys (sorted vertex ids)
    struct HF {
      std::array<int64_t, 3> key;
      int64_t c;
      int f;
    };
    std::vector<HF> hf(nc * nf);
    for (int64_t c = 0; c < nc; ++c)
      for (int f = 0; f < nf; ++f) {
        HF& x = hf[c * nf + f];
        x.key = {-1, -1, -1};
        int t = 0;
        for (int v = 0; v < nf; ++v)
          if (v != f) x.key[t++] = M.cells[c * nf + v];
        std::sort(x.key.begin(), x.key.begin() + dim);
        x.c = c;
        x.f = f;
      }
    std::sort(hf.begin(), hf.end(), [](const HF& a, const HF& b) {
      if (a.key != b.key) return a.key < b.key;
      return a.c < b.c;
    });
    w.sib.assign(nc * nf, -1);
    w.sib_f.assign(nc * nf, -1);
    for (size_t i = 0; i < hf.size();) {
      size_t j = i + 1;
      while (j < hf.size() && hf[j].key == hf[i].key) ++j;
      if (j - i > 2) {
        *err = "mesh " + std::to_string(k) + ": a facet is shared by more than two cells";
        return WLSENO_ERR_MESH;
      }
      if (j - i == 2) {
        if (hf[i].c == hf[i + 1].c) {
          *err = "mesh " + std::to_string(k) + ": a cell repeats a vertex";
          return WLSENO_ERR_MESH;
        }
        w.sib[hf[i].c * nf + hf[i].f] = hf[i + 1].c;
        w.sib_f[hf[i].c * nf + hf[i].f] = static_cast<int8_t>(hf[i + 1].f);
        w.sib[hf[i + 1].c * nf + hf[i + 1].f] = hf[i].c;
        w.sib_f[hf[i + 1].c * nf + hf[i + 1].f] = static_cast<int8_t>(hf[i].f);
      }
      i = j;
    }
    // ---- facet data: owner-oriented normal/area, neighbours, quadrature points
    const double g = std::sqrt(3.0) / 6.0;
    for (int64_t c = 0; c < nc; ++c) {
      const int64_t gc = base + c;
      const double* X = &S.coords[gc * nf * dim];
      for (int f = 0; f < nf; ++f) {
        int64_t s = w.sib[c * nf + f];
        int64_t owner = (s < 0 || c < s) ? c : s;
        int owner_f = (owner == c) ? f : w.sib_f[c * nf + f];
        int64_t gowner = base + owner;
        double* G = &S.fgeo[(gc * nf + f) * 4];
        for (int a = 0; a < dim; ++a) G[a] = own_normal[(gowner * nf + owner_f) * 3 + a];
        G[3] = own_area[gowner * nf + owner_f];
        if (s >= 0) S.nbr[gc * nf + f] = static_cast<int32_t>(((base + s) << 2) | w.sib_f[c * nf + f]);
        // facet vertices (local slots) sorted by global vertex index
        int loc[3], t = 0;
        for (int v = 0; v < nf; ++v)
          if (v != f) loc[t++] = v;
        std::sort(loc, loc + dim,
                  [&](int a, int b) { return M.cells[c * nf + a] < M.cells[c * nf + b]; });
        for (int q = 0; q < nq; ++q) {
          double bary[3];
          if (dim == 1) {
            bary[0] = 1.0;
          } else if (dim == 2) {
            double tq = q == 0 ? 0.5 - g : 0.5 + g;
            bary[0] = 1.0 - tq;
            bary[1] = tq;
          } else {
            for (int a = 0; a < 3; ++a) bary[a] = (a == q) ? 2.0 / 3.0 : 1.0 / 6.0;
          }
          for (int a = 0; a < dim; ++a) {
            double x = 0.0;
            for (int b = 0; b < dim; ++b) x += bary[b] * X[loc[b] * dim + a];
            S.fpts[((gc * nf + f) * nq + q) * dim + a] = (x - S.centroid[gc * dim + a]) / S.h[gc];
          }
        }
      }
    }
    // ---- k-ring stencils
    std::vector<int64_t> stamp(nc, -1);
    std::vector<int64_t> set, grown, outer;
    std::vector<int> outer_steps(static_cast<int>(std::floor(opts->ring + 1e-9)) + 1, kVertex);
    const std::vector<int> bal_steps(std::max(balance_steps, 0), kVertex);
    auto add = [&](int64_t x, int64_t tag, std::vector<int64_t>& into) {
      if (stamp[x] != tag) {
        stamp[x] = tag;
        into.push_back(x);
      }
    };
    int64_t tag = 0;
    auto grow = [&](const std::vector<int>& st, int64_t c) {
      // returns the ring in `set`; stamps of members == current tag
      ++tag;
      set.clear();
      add(c, tag, set);
      for (int kind : st) {
        size_t cur = set.size();
        for (size_t t = 0; t < cur; ++t) {
          int64_t x = set[t];
          const int64_t* cv = M.cells + x * nf;
          if (kind == kFacet) {
            for (int f = 0; f < nf; ++f) {
              int64_t y = w.sib[x * nf + f];
              if (y >= 0) add(y, tag, set);
            }
          } else if (kind == kVertex) {
            for (int v = 0; v < nf; ++v)
              for (int64_t q = w.inc_ptr[cv[v]]; q < w.inc_ptr[cv[v] + 1]; ++q) add(w.inc[q], tag, set);
          } else {
            for (int a = 0; a < nf; ++a)
              for (int b = a + 1; b < nf; ++b)
                for_cells_sharing_edge(w, cv[a], cv[b], [&](int64_t y) { add(y, tag, set); });
          }
        }
      }
    };
    const double cut = opts->radius_cut;
    for (int64_t c = 0; c < nc; ++c) {
      const int64_t gc = base + c;
      std::vector<int64_t> members;
      if (cut > 0.0) {
        grow(outer_steps, c);
        outer = set;
      }
      grow(steps, c);
      members = set;
      int64_t mtag = tag;
      if (cut > 0.0) {
        for (int64_t y : outer) {
          if (stamp[y] == mtag) continue;
          double d2 = 0.0;
          for (int a = 0; a < dim; ++a) {
            double d = wrap_delta(S.centroid[(base + y) * dim + a] - S.centroid[gc * dim + a], L[a]);
            d2 += d * d;
          }
          if (std::sqrt(d2) <= cut * S.h[gc]) {
            stamp[y] = mtag;
            members.push_back(y);
          }
        }
      }
      while (static_cast<int>(members.size()) < min_rows) {
        size_t before = members.size();
        for (size_t t = 0; t < before; ++t)
          for (int f = 0; f < nf; ++f) {
            int64_t y = w.sib[members[t] * nf + f];
            if (y >= 0 && stamp[y] != mtag) {
              stamp[y] = mtag;
              members.push_back(y);
            }
          }
        if (members.size() == before) break;
      }
      // facet neighbours must belong to the stencil (beta of the centre)
      for (int f = 0; f < nf; ++f) {
        int64_t y = w.sib[c * nf + f];
        if (y >= 0 && stamp[y] != mtag) {
          *err = "facet neighbour outside the stencil";
          return WLSENO_ERR_STENCIL;
        }
      }
      std::sort(members.begin() + 1, members.end());
      if (static_cast<int>(members.size()) < m) {
        *err = "mesh " + std::to_string(k) + ": cell " + std::to_string(c) + " has a stencil of " +
               std::to_string(members.size()) + " cells < m = " + std::to_string(m);
        return WLSENO_ERR_STENCIL;
      }
      S.row_ptr[gc + 1] = static_cast<int64_t>(members.size());
      for (int64_t y : members) S.cols.push_back(base + y);
      if (balance_steps > 0) {
        grow(bal_steps, c);
        std::sort(set.begin() + 1, set.end());
        S.bal_ptr[gc + 1] = static_cast<int64_t>(set.size()) - 1;
        for (size_t t = 1; t < set.size(); ++t) S.bal_idx.push_back(base + set[t]);
      }
    }
    base += nc;
  }
  for (int64_t i = 0; i < N; ++i) S.row_ptr[i + 1] += S.row_ptr[i];
  if (balance_steps > 0) {
    for (int64_t i = 0; i < N; ++i) S.bal_ptr[i + 1] += S.bal_ptr[i];
    if (S.bal_ptr[N] >= (int64_t(1) << 31)) {
      *err = "balanced-stencil candidates exceed 32-bit offsets";
      return WLSENO_ERR_STENCIL;
    }
  }
  S.nnz = S.row_ptr[N];
  S.max_n = 0;
  S.min_n = 1 << 30;
  for (int64_t i = 0; i < N; ++i) {
    int n = static_cast<int>(S.row_ptr[i + 1] - S.row_ptr[i]);
    S.max_n = std::max(S.max_n, n);
    S.min_n = std::min(S.min_n, n);
  }
  // transposed stencils for the adjoint's deterministic gather
  S.tr_ptr.assign(N + 1, 0);
  for (int64_t c = 0; c < N; ++c)
    for (int64_t e = S.row_ptr[c] + 1; e < S.row_ptr[c + 1]; ++e) S.tr_ptr[S.cols[e] + 1]++;
  for (int64_t j = 0; j < N; ++j) S.tr_ptr[j + 1] += S.tr_ptr[j];
  S.tr_slot.assign(S.tr_ptr[N], 0);
  {
    std::vector<int64_t> fill(S.tr_ptr.begin(), S.tr_ptr.end() - 1);
    for (int64_t c = 0; c < N; ++c)
      for (int64_t e = S.row_ptr[c] + 1; e < S.row_ptr[c + 1]; ++e)
        S.tr_slot[fill[S.cols[e]]++] = (e - S.row_ptr[c]) * N + c;  // ascending c, then t
  }
  if (S.nnz >= (int64_t(1) << 31)) {
    *err = "stencil storage exceeds 32-bit offsets";
    return WLSENO_ERR_STENCIL;
  }
  return WLSENO_OK;
}

}  // namespace wlseno
