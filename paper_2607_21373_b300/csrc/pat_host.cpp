// Host-side FP64 assembly of the P1 operators, sensor location and the
// time-step growth check (Section 3 of arXiv 2607.21373).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <unordered_map>

#include "pat_internal.h"

namespace pat {

namespace {
thread_local std::string g_err;
}

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

// Element volume and barycentric gradients: with J = [X1-X0, X2-X0, X3-X0]
// (columns), grad l_a is row a of J^{-1} for a = 1..3, grad l_0 = -sum.
static double tet_geometry(const double* X0, const double* X1, const double* X2, const double* X3,
                           double g[4][3]) {
  double J[3][3];
  for (int r = 0; r < 3; ++r) {
    J[r][0] = X1[r] - X0[r];
    J[r][1] = X2[r] - X0[r];
    J[r][2] = X3[r] - X0[r];
  }
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (det == 0.0) return 0.0;
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int c = 0; c < 3; ++c) {
    g[1][c] = inv[0][c];
    g[2][c] = inv[1][c];
    g[3][c] = inv[2][c];
    g[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
  }
  return std::fabs(det) / 6.0;
}

// CSR pattern of the node graph of a set of cliques (tets: 4, faces: 3).
static void clique_pattern(int64_t N, const int32_t* cl, int64_t n_cl, int w, std::vector<int64_t>& ptr,
                           std::vector<int32_t>& col) {
  std::vector<int64_t> cnt(N + 1, 0);
  for (int64_t e = 0; e < n_cl; ++e)
    for (int a = 0; a < w; ++a) cnt[cl[e * w + a] + 1] += w;
  std::vector<int64_t> start(N + 1, 0);
  for (int64_t i = 0; i < N; ++i) start[i + 1] = start[i] + cnt[i + 1];
  std::vector<int32_t> tmp(start[N]);
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t e = 0; e < n_cl; ++e)
    for (int a = 0; a < w; ++a)
      for (int b = 0; b < w; ++b) tmp[fill[cl[e * w + a]]++] = cl[e * w + b];
  ptr.assign(N + 1, 0);
  col.clear();
  col.reserve(start[N] / 3 + N);
  for (int64_t i = 0; i < N; ++i) {
    auto b = tmp.begin() + start[i], en = tmp.begin() + start[i + 1];
    std::sort(b, en);
    auto u = std::unique(b, en);
    col.insert(col.end(), b, u);
    ptr[i + 1] = static_cast<int64_t>(col.size());
  }
}

static inline int64_t find_col(const std::vector<int64_t>& ptr, const std::vector<int32_t>& col, int64_t i,
                               int32_t j) {
  auto b = col.begin() + ptr[i], e = col.begin() + ptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  return (it != e && *it == j) ? (it - col.begin()) : -1;
}

void assemble_stiffness(HostMesh& m) {
  m.k_val.assign(m.k_col.size(), 0.0);
  m.ml.assign(m.N, 0.0);
  for (int64_t e = 0; e < m.E; ++e) {
    const int32_t* t = &m.tets[4 * e];
    const double* g = &m.grads[e * 12];
    const double s = m.c2[e] * m.vol[e];
    for (int a = 0; a < 4; ++a) {
      m.ml[t[a]] += m.vol[e] / 4.0;  // row sum of the consistent P1 mass V/20 (1 + delta_ab)
      for (int b = 0; b < 4; ++b) {
        const double v = s * (g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2]);
        m.k_val[find_col(m.k_ptr, m.k_col, t[a], t[b])] += v;
      }
    }
  }
}

pat_status assemble_host(const double* xyz, int64_t N, const int32_t* tets, int64_t E, const double* c2,
                         HostMesh& m) {
  if (N < 4 || E < 1) {
    set_error("pat_mesh_create: need at least 4 nodes and 1 tetrahedron (got %lld, %lld)", (long long)N,
              (long long)E);
    return PAT_EINVAL;
  }
  if (N >= (int64_t)kIdxMask) {
    set_error("pat_mesh_create: too many nodes (%lld)", (long long)N);
    return PAT_EINVAL;
  }
  m.N = N;
  m.E = E;
  m.xyz.assign(xyz, xyz + 3 * N);
  m.tets.assign(tets, tets + 4 * E);
  m.c2.assign(E, 1.0);
  if (c2) m.c2.assign(c2, c2 + E);
  for (int64_t e = 0; e < 4 * E; ++e) {
    if (tets[e] < 0 || tets[e] >= N) {
      set_error("pat_mesh_create: tetrahedron %lld has vertex %d outside [0, %lld)", (long long)(e / 4), tets[e],
                (long long)N);
      return PAT_EINVAL;
    }
  }
  for (int64_t e = 0; e < E; ++e) {
    if (!(m.c2[e] > 0.0) || !std::isfinite(m.c2[e])) {
      set_error("pat_mesh_create: c2 of tetrahedron %lld is %g (must be finite and > 0)", (long long)e, m.c2[e]);
      return PAT_EINVAL;
    }
  }
  // bounding box for the relative degeneracy tolerance
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], xyz[3 * i + c]);
      hi[c] = std::max(hi[c], xyz[3 * i + c]);
    }
  double diam = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                          (hi[2] - lo[2]) * (hi[2] - lo[2]));
  m.vol.resize(E);
  m.grads.resize(E * 12);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* t = tets + 4 * e;
    double g[4][3];
    double V = tet_geometry(xyz + 3 * t[0], xyz + 3 * t[1], xyz + 3 * t[2], xyz + 3 * t[3], g);
    // a tetrahedron whose volume is 1e-12 of the bounding box volume is degenerate
    if (!(V > 1e-12 * diam * diam * diam / std::max<int64_t>(E, 1))) {
      set_error("pat_mesh_create: tetrahedron %lld is degenerate (volume %g)", (long long)e, V);
      return PAT_EINVAL;
    }
    m.vol[e] = V;
    std::memcpy(&m.grads[e * 12], g, sizeof(g));
  }
  // stiffness K_e = c^2 V grad l_a . grad l_b on the full P1 graph
  clique_pattern(N, tets, E, 4, m.k_ptr, m.k_col);
  assemble_stiffness(m);
  for (int64_t i = 0; i < N; ++i) {
    if (!(m.ml[i] > 0.0)) {
      set_error("pat_mesh_create: node %lld belongs to no tetrahedron", (long long)i);
      return PAT_EINVAL;
    }
  }
  // boundary faces: triangles seen by exactly one tetrahedron
  std::vector<std::array<int32_t, 3>> faces;
  faces.reserve(4 * E);
  static const int fidx[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* t = tets + 4 * e;
    for (int f = 0; f < 4; ++f) {
      std::array<int32_t, 3> tri = {t[fidx[f][0]], t[fidx[f][1]], t[fidx[f][2]]};
      std::sort(tri.begin(), tri.end());
      faces.push_back(tri);
    }
  }
  std::sort(faces.begin(), faces.end());
  m.bfaces.clear();
  for (size_t i = 0; i < faces.size();) {
    size_t j = i;
    while (j < faces.size() && faces[j] == faces[i]) ++j;
    if (j - i == 1) m.bfaces.insert(m.bfaces.end(), faces[i].begin(), faces[i].end());
    if (j - i > 2) {
      set_error("pat_mesh_create: a triangle is shared by %zu tetrahedra (non-manifold mesh)", j - i);
      return PAT_EINVAL;
    }
    i = j;
  }
  int64_t F = (int64_t)m.bfaces.size() / 3;
  if (F == 0) {
    set_error("pat_mesh_create: mesh has no boundary triangles");
    return PAT_EINVAL;
  }
  clique_pattern(N, m.bfaces.data(), F, 3, m.b_ptr, m.b_col);
  m.b_val.assign(m.b_col.size(), 0.0);
  for (int64_t f = 0; f < F; ++f) {
    const int32_t* t = &m.bfaces[3 * f];
    const double *P0 = &xyz[3 * t[0]], *P1 = &xyz[3 * t[1]], *P2 = &xyz[3 * t[2]];
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
      e1[c] = P1[c] - P0[c];
      e2[c] = P2[c] - P0[c];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
    double A = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        m.b_val[find_col(m.b_ptr, m.b_col, t[a], t[b])] += (A / 12.0) * (a == b ? 2.0 : 1.0);
  }
  m.n_boundary_nodes = 0;
  for (int64_t i = 0; i < N; ++i) m.n_boundary_nodes += (m.b_ptr[i + 1] > m.b_ptr[i]);
  return PAT_OK;
}

// Sensor location: uniform grid over the boundary triangles' bounding boxes;
// a sensor is accepted by a triangle when its distance to the triangle's plane
// is below 1e-9 of the triangle size and all barycentric coordinates are
// >= -1e-12; among several, the largest minimum coordinate wins (lowest
// triangle index on ties).
// Sensors inside the mesh (neither a node nor on a boundary triangle): the
// tetrahedron that holds the point and its four barycentric coordinates (P1
// interpolation).  Tetrahedra are hashed by their bounding boxes on a uniform
// grid of the largest tetrahedron extent, built on the first such sensor.
struct TetGrid {
  bool built = false;
  double lo[3] = {0, 0, 0}, cell = 1.0;
  int64_t dims[3] = {1, 1, 1};
  std::unordered_map<int64_t, std::vector<int32_t>> cells;
};

static void build_tet_grid(const HostMesh& m, TetGrid& g) {
  const double* X = m.xyz.data();
  double hi[3] = {-1e300, -1e300, -1e300}, hmax = 0.0;
  for (int c = 0; c < 3; ++c) g.lo[c] = 1e300;
  for (int64_t i = 0; i < m.N; ++i)
    for (int c = 0; c < 3; ++c) {
      g.lo[c] = std::min(g.lo[c], X[3 * i + c]);
      hi[c] = std::max(hi[c], X[3 * i + c]);
    }
  for (int64_t e = 0; e < m.E; ++e)
    for (int c = 0; c < 3; ++c) {
      double a = 1e300, b = -1e300;
      for (int v = 0; v < 4; ++v) {
        const double t = X[3 * (int64_t)m.tets[4 * e + v] + c];
        a = std::min(a, t);
        b = std::max(b, t);
      }
      hmax = std::max(hmax, b - a);
    }
  g.cell = std::max(hmax, 1e-300);
  for (int c = 0; c < 3; ++c) g.dims[c] = std::max<int64_t>(1, (int64_t)std::ceil((hi[c] - g.lo[c]) / g.cell) + 1);
  for (int64_t e = 0; e < m.E; ++e) {
    int64_t a0[3], a1[3];
    for (int c = 0; c < 3; ++c) {
      double a = 1e300, b = -1e300;
      for (int v = 0; v < 4; ++v) {
        const double t = X[3 * (int64_t)m.tets[4 * e + v] + c];
        a = std::min(a, t);
        b = std::max(b, t);
      }
      a0[c] = std::min(std::max<int64_t>((int64_t)std::floor((a - g.lo[c]) / g.cell), 0), g.dims[c] - 1);
      a1[c] = std::min(std::max<int64_t>((int64_t)std::floor((b - g.lo[c]) / g.cell), 0), g.dims[c] - 1);
    }
    for (int64_t i = a0[0]; i <= a1[0]; ++i)
      for (int64_t j = a0[1]; j <= a1[1]; ++j)
        for (int64_t k = a0[2]; k <= a1[2]; ++k)
          g.cells[(i * g.dims[1] + j) * g.dims[2] + k].push_back((int32_t)e);
  }
  g.built = true;
}

static pat_status locate_in_tets(const double* x, int32_t d, HostMesh& m, TetGrid& g) {
  if (!g.built) build_tet_grid(m, g);
  const double* X = m.xyz.data();
  int64_t ijk[3];
  for (int c = 0; c < 3; ++c) {
    const int64_t v = (int64_t)std::floor((x[c] - g.lo[c]) / g.cell);
    if (v < 0 || v >= g.dims[c]) {
      set_error("pat_mesh_create: sensor %d at (%g, %g, %g) is outside the mesh", d, x[0], x[1], x[2]);
      return PAT_EINVAL;
    }
    ijk[c] = v;
  }
  auto it = g.cells.find((ijk[0] * g.dims[1] + ijk[1]) * g.dims[2] + ijk[2]);
  int64_t best = -1;
  double best_min = -1e300, best_l[4] = {0, 0, 0, 0};
  if (it != g.cells.end())
    for (int32_t e : it->second) {
      const int32_t* t = &m.tets[4 * (int64_t)e];
      const double* P0 = X + 3 * (int64_t)t[0];
      double J[3][3], r[3];
      for (int c = 0; c < 3; ++c) {
        for (int v = 0; v < 3; ++v) J[c][v] = X[3 * (int64_t)t[v + 1] + c] - P0[c];
        r[c] = x[c] - P0[c];
      }
      // solve J l = r by Cramer's rule (J's columns are the edges from vertex 0)
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      if (det == 0.0) continue;
      double l[4];
      for (int v = 0; v < 3; ++v) {
        double A[3][3];
        for (int c = 0; c < 3; ++c)
          for (int u = 0; u < 3; ++u) A[c][u] = (u == v) ? r[c] : J[c][u];
        l[v + 1] = (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) /
                   det;
      }
      l[0] = 1.0 - l[1] - l[2] - l[3];
      const double mn = std::min(std::min(l[0], l[1]), std::min(l[2], l[3]));
      if (mn < -1e-12) continue;
      if (mn > best_min || (mn == best_min && e < best)) {
        best = e;
        best_min = mn;
        for (int v = 0; v < 4; ++v) best_l[v] = l[v];
      }
    }
  if (best < 0) {
    set_error("pat_mesh_create: sensor %d at (%g, %g, %g) is not inside the mesh", d, x[0], x[1], x[2]);
    return PAT_EINVAL;
  }
  double s = 0.0;
  for (int v = 0; v < 4; ++v) {
    best_l[v] = std::max(best_l[v], 0.0);
    s += best_l[v];
  }
  for (int v = 0; v < 4; ++v) {
    m.det_node[kDetPts * d + v] = m.tets[4 * best + v];
    m.det_w[kDetPts * d + v] = best_l[v] / s;
  }
  return PAT_OK;
}

pat_status locate_sensors(const double* det, int32_t n_obs, HostMesh& m) {
  TetGrid tet_grid;
  const int64_t F = (int64_t)m.bfaces.size() / 3;
  const double* X = m.xyz.data();
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double hmax = 0.0;
  for (int64_t f = 0; f < F; ++f) {
    double flo[3] = {1e300, 1e300, 1e300}, fhi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        double v = X[3 * m.bfaces[3 * f + a] + c];
        flo[c] = std::min(flo[c], v);
        fhi[c] = std::max(fhi[c], v);
      }
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], flo[c]);
      hi[c] = std::max(hi[c], fhi[c]);
      hmax = std::max(hmax, fhi[c] - flo[c]);
    }
  }
  const double cell = std::max(hmax, 1e-300);
  int64_t dims[3];
  for (int c = 0; c < 3; ++c) dims[c] = std::max<int64_t>(1, (int64_t)std::ceil((hi[c] - lo[c]) / cell) + 1);
  auto cell_of = [&](const double* p, int64_t ijk[3]) {
    for (int c = 0; c < 3; ++c) {
      int64_t v = (int64_t)std::floor((p[c] - lo[c]) / cell);
      ijk[c] = std::min(std::max<int64_t>(v, 0), dims[c] - 1);
    }
  };
  std::unordered_map<int64_t, std::vector<int32_t>> grid;
  for (int64_t f = 0; f < F; ++f) {
    double flo[3] = {1e300, 1e300, 1e300}, fhi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        double v = X[3 * m.bfaces[3 * f + a] + c];
        flo[c] = std::min(flo[c], v);
        fhi[c] = std::max(fhi[c], v);
      }
    int64_t a0[3], a1[3];
    cell_of(flo, a0);
    cell_of(fhi, a1);
    for (int64_t i = a0[0]; i <= a1[0]; ++i)
      for (int64_t j = a0[1]; j <= a1[1]; ++j)
        for (int64_t k = a0[2]; k <= a1[2]; ++k) grid[(i * dims[1] + j) * dims[2] + k].push_back((int32_t)f);
  }
  m.n_obs = n_obs;
  m.det_node.assign(kDetPts * (size_t)n_obs, 0);
  m.det_w.assign(kDetPts * (size_t)n_obs, 0.0);
  // node-coincident sensors (any node, interior ones included): nodes hashed by
  // their coordinates quantised to q = 1e-9 of the mesh's extent; a sensor
  // within 1e-12 of the extent of a node observes that node's value alone
  double ext = 0.0, nlo[3] = {1e300, 1e300, 1e300};
  for (int64_t i = 0; i < m.N; ++i)
    for (int c = 0; c < 3; ++c) nlo[c] = std::min(nlo[c], X[3 * i + c]);
  for (int64_t i = 0; i < m.N; ++i)
    for (int c = 0; c < 3; ++c) ext = std::max(ext, X[3 * i + c] - nlo[c]);
  const double q = std::max(ext, 1e-300) * 1e-9;
  auto qkey = [&](const double* p, int di, int dj, int dk) {
    const int64_t a = (int64_t)std::floor((p[0] - nlo[0]) / q) + di, b = (int64_t)std::floor((p[1] - nlo[1]) / q) + dj,
                  c = (int64_t)std::floor((p[2] - nlo[2]) / q) + dk;
    return (uint64_t)(a * 73856093LL) ^ (uint64_t)(b * 19349663LL) ^ (uint64_t)(c * 83492791LL);
  };
  std::unordered_multimap<uint64_t, int32_t> node_hash;
  node_hash.reserve((size_t)m.N);
  for (int64_t i = 0; i < m.N; ++i) node_hash.emplace(qkey(X + 3 * i, 0, 0, 0), (int32_t)i);
  auto node_at = [&](const double* p) -> int32_t {
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj)
        for (int dk = -1; dk <= 1; ++dk) {
          auto range = node_hash.equal_range(qkey(p, di, dj, dk));
          for (auto it = range.first; it != range.second; ++it) {
            const double* y = X + 3 * (int64_t)it->second;
            if (std::fabs(y[0] - p[0]) <= 1e-12 * ext && std::fabs(y[1] - p[1]) <= 1e-12 * ext &&
                std::fabs(y[2] - p[2]) <= 1e-12 * ext)
              return it->second;
          }
        }
    return -1;
  };
  for (int32_t d = 0; d < n_obs; ++d) {
    const double* x = det + 3 * d;
    const int32_t at = node_at(x);
    if (at >= 0) {
      for (int a = 0; a < kDetPts; ++a) {
        m.det_node[kDetPts * d + a] = at;
        m.det_w[kDetPts * d + a] = a == 0 ? 1.0 : 0.0;
      }
      continue;
    }
    int64_t c0[3];
    cell_of(x, c0);
    int64_t best = -1;
    double best_min = -1e300, best_l[3] = {0, 0, 0};
    for (int64_t i = std::max<int64_t>(0, c0[0] - 1); i <= std::min(dims[0] - 1, c0[0] + 1); ++i)
      for (int64_t j = std::max<int64_t>(0, c0[1] - 1); j <= std::min(dims[1] - 1, c0[1] + 1); ++j)
        for (int64_t k = std::max<int64_t>(0, c0[2] - 1); k <= std::min(dims[2] - 1, c0[2] + 1); ++k) {
          auto it = grid.find((i * dims[1] + j) * dims[2] + k);
          if (it == grid.end()) continue;
          for (int32_t f : it->second) {
            const int32_t* t = &m.bfaces[3 * f];
            const double *P0 = X + 3 * t[0], *P1 = X + 3 * t[1], *P2 = X + 3 * t[2];
            double e1[3], e2[3], r[3];
            for (int c = 0; c < 3; ++c) {
              e1[c] = P1[c] - P0[c];
              e2[c] = P2[c] - P0[c];
              r[c] = x[c] - P0[c];
            }
            double n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2],
                   n2 = e1[0] * e2[1] - e1[1] * e2[0];
            double nn = std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
            double size = std::sqrt(std::max(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2],
                                             e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]));
            double dist = std::fabs(n0 * r[0] + n1 * r[1] + n2 * r[2]) / nn;
            if (dist > 1e-9 * size) continue;
            double g11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
            double g12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
            double g22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
            double r1 = e1[0] * r[0] + e1[1] * r[1] + e1[2] * r[2];
            double r2 = e2[0] * r[0] + e2[1] * r[1] + e2[2] * r[2];
            double det2 = g11 * g22 - g12 * g12;
            double l1 = (g22 * r1 - g12 * r2) / det2;
            double l2 = (g11 * r2 - g12 * r1) / det2;
            double l0 = 1.0 - l1 - l2;
            double mn = std::min(l0, std::min(l1, l2));
            if (mn < -1e-12) continue;
            if (mn > best_min || (mn == best_min && f < best)) {
              best = f;
              best_min = mn;
              best_l[0] = l0;
              best_l[1] = l1;
              best_l[2] = l2;
            }
          }
        }
    if (best < 0) {
      const pat_status si = locate_in_tets(x, d, m, tet_grid);
      if (si) return si;
      continue;
    }
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
      best_l[a] = std::max(best_l[a], 0.0);
      s += best_l[a];
    }
    for (int a = 0; a < 3; ++a) {
      m.det_node[kDetPts * d + a] = m.bfaces[3 * best + a];
      m.det_w[kDetPts * d + a] = best_l[a] / s;
    }
    m.det_node[kDetPts * d + 3] = m.bfaces[3 * best];  // unused fourth point: weight 0
  }
  return PAT_OK;
}

// Runs the FP64 propagator (p, v form of eq. fully-discrete with M_L) from a
// seeded random state for 300 steps; the growth factor over the last 200 steps
// is compared with 100 (a spectral radius above ~1.023).  The norm is the
// energy-like sqrt(v^T M_L v + p^T M_L p / T^2) rescaled every step.
pat_status check_stability(const HostMesh& m, double* growth_out) {
  const int64_t N = m.N;
  const double dt = m.dt;
  std::vector<double> p(N), v(N), ph(N), kp(N), bv(N);
  std::mt19937_64 rng(12345);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int64_t i = 0; i < N; ++i) {
    p[i] = nd(rng);
    v[i] = nd(rng);
  }
  // drop exact zeros once for speed
  std::vector<int64_t> kp_ptr(N + 1, 0);
  std::vector<int32_t> kc;
  std::vector<double> kv;
  for (int64_t i = 0; i < N; ++i) {
    for (int64_t e = m.k_ptr[i]; e < m.k_ptr[i + 1]; ++e)
      if (m.k_val[e] != 0.0) {
        kc.push_back(m.k_col[e]);
        kv.push_back(m.k_val[e]);
      }
    kp_ptr[i + 1] = (int64_t)kc.size();
  }
  auto norm = [&]() {
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += m.ml[i] * (v[i] * v[i] + p[i] * p[i] / (dt * dt));
    return std::sqrt(s);
  };
  double log_growth = 0.0;
  double n0 = norm();
  for (int step = 0; step < 300; ++step) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) ph[i] = p[i] + 0.5 * dt * v[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      double s = 0.0, b = 0.0;
      for (int64_t e = kp_ptr[i]; e < kp_ptr[i + 1]; ++e) s += kv[e] * ph[kc[e]];
      for (int64_t e = m.b_ptr[i]; e < m.b_ptr[i + 1]; ++e) b += m.b_val[e] * v[m.b_col[e]];
      kp[i] = s;
      bv[i] = b;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
      v[i] = v[i] - dt * (kp[i] + bv[i]) / m.ml[i];
      p[i] = ph[i] + 0.5 * dt * v[i];
    }
    double n1 = norm();
    if (!std::isfinite(n1)) {
      log_growth = 1e300;
      break;
    }
    if (step >= 100) log_growth += std::log(n1 / n0);
    for (int64_t i = 0; i < N; ++i) {
      p[i] /= n1;
      v[i] /= n1;
    }
    n0 = 1.0;
  }
  double growth = std::exp(std::min(log_growth, 700.0));
  if (growth_out) *growth_out = growth;
  if (!(growth <= 100.0)) {
    set_error("pat_mesh_create: dt = %g is unstable: the propagator grew by %g over 200 steps "
              "(spectral radius > 1); reduce dt",
              dt, growth);
    return PAT_EUNSTABLE;
  }
  return PAT_OK;
}

}  // namespace pat
