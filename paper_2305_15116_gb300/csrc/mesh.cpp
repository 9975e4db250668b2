// Host mesh module: coarse topology, uniform refinement bookkeeping, the
// per-macro constant stencils and the kernels' work lists.
//
// Sec. 1.2 of the paper: the coarse mesh is unstructured, every macro is
// refined uniformly, and inside a macro all rows of the matrix are the same
// stencil because the refinement is affine.  The stencil of a macro is the sum
// of the P1 element matrices of the micro-elements around a point; this file
// computes it once per macro and level, together with the partial stencils of
// points on the macro's own edges/faces/vertices (only the micro-elements of
// this macro), which the interface kernel sums over all incident macros.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <numeric>

#include "hyteg_internal.h"

namespace hyteg {

namespace {

const int OFF2[NW2][2] = {{0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}};
const int OFF3[NW3][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                          {1, -1, 0}, {-1, 1, 0},  {0, 0, 1},  {-1, 0, 1},  {0, -1, 1},
                          {1, -1, 1}, {0, 0, -1},  {1, 0, -1}, {0, 1, -1},  {-1, 1, -1}};

int find_off2(int dx, int dy) {
  for (int k = 0; k < NW2; ++k)
    if (OFF2[k][0] == dx && OFF2[k][1] == dy) return k;
  return -1;
}
int find_off3(int dx, int dy, int dz) {
  for (int k = 0; k < NW3; ++k)
    if (OFF3[k][0] == dx && OFF3[k][1] == dy && OFF3[k][2] == dz) return k;
  return -1;
}

// Micro-element types as vertex offsets in the macro's index space.
// 2D: the "up" and "down" triangles of the regular refinement.
const int ELEM2[2][3][2] = {{{0, 0}, {1, 0}, {0, 1}}, {{1, 0}, {0, 1}, {1, 1}}};

// 3D: the Kuhn simplices.  In the coordinates u = (x+y+z, y+z, z) the unit
// cube splits into six simplices a, a+e_p, a+e_p+e_q, a+(1,1,1), one per axis
// permutation (p,q,r).  Mapped back (x = u1-u2, y = u2-u3, z = u3) they tile a
// refined macro-tet with n^3 elements.
void kuhn_types(int out[6][4][3]) {
  int perm[3] = {0, 1, 2};
  int t = 0;
  do {
    int u[4][3] = {{0, 0, 0}};
    for (int s = 1; s < 4; ++s) {
      for (int c = 0; c < 3; ++c) u[s][c] = u[s - 1][c];
      u[s][perm[s - 1]] += 1;
    }
    for (int s = 0; s < 4; ++s) {
      out[t][s][0] = u[s][0] - u[s][1];
      out[t][s][1] = u[s][1] - u[s][2];
      out[t][s][2] = u[s][2];
    }
    ++t;
  } while (std::next_permutation(perm, perm + 3));
}

// P1 Laplace element matrix of a triangle by the cotangent formula: the
// coupling of vertices i and j is -cot(angle at the third vertex k) / 2 and
// every row sums to zero.
void tri_stiffness(const double P[3][2], double K[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K[i][j] = 0.0;
  for (int k = 0; k < 3; ++k) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    const double ax = P[i][0] - P[k][0], ay = P[i][1] - P[k][1];
    const double bx = P[j][0] - P[k][0], by = P[j][1] - P[k][1];
    const double cot = (ax * bx + ay * by) / std::fabs(ax * by - ay * bx);
    K[i][j] = K[j][i] = -0.5 * cot;
  }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      if (j != i) s += K[i][j];
    K[i][i] = -s;
  }
}

// P1 Laplace element matrix of a tetrahedron: K_ab = |T| grad(l_a).grad(l_b),
// barycentric gradients from the inverse of the edge matrix (adjugate / det).
void tet_stiffness(const double P[4][3], double K[4][4]) {
  double J[3][3];  // columns: P1-P0, P2-P0, P3-P0
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) J[r][c] = P[c + 1][r] - P[0][r];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  // rows of J^{-1} are the gradients of l_1, l_2, l_3
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
  double g[4][3];
  for (int c = 0; c < 3; ++c) {
    g[1][c] = inv[0][c];
    g[2][c] = inv[1][c];
    g[3][c] = inv[2][c];
    g[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
  }
  const double vol = std::fabs(det) / 6.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) K[a][b] = vol * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
}

// Does an offset d from a point of boundary class `cls` stay inside the macro?
// 2D class bits: 0 x=0, 1 y=0, 2 x+y=n.  3D: 0 x=0, 1 y=0, 2 z=0, 3 x+y+z=n.
bool inside2(int cls, int dx, int dy) {
  if ((cls & 1) && dx < 0) return false;
  if ((cls & 2) && dy < 0) return false;
  if ((cls & 4) && dx + dy > 0) return false;
  return true;
}
bool inside3(int cls, int dx, int dy, int dz) {
  if ((cls & 1) && dx < 0) return false;
  if ((cls & 2) && dy < 0) return false;
  if ((cls & 4) && dz < 0) return false;
  if ((cls & 8) && dx + dy + dz > 0) return false;
  return true;
}

template <class T>
std::string upload(const Mesh& m, T** dptr, const std::vector<T>& h) {
  if (h.empty()) {
    *dptr = nullptr;
    return "";
  }
  cudaError_t e = dev_alloc(m, (void**)dptr, h.size() * sizeof(T));
  if (e != cudaSuccess) {
    *dptr = nullptr;
    return std::string("device allocation: ") + cudaGetErrorString(e);
  }
  e = dev_upload(m, *dptr, h.data(), h.size() * sizeof(T));
  if (e != cudaSuccess) return std::string("host-to-device copy: ") + cudaGetErrorString(e);
  return "";
}

}  // namespace

int64_t slots_per_macro(int dim, int level) {
  const int64_t n = int64_t(1) << level;
  return dim == 2 ? (n + 1) * (n + 2) / 2 : (n + 1) * (n + 2) * (n + 3) / 6;
}

int64_t n_global_dofs(const Mesh& m, int level) {
  const int64_t n = int64_t(1) << level;
  const int64_t ne = std::max<int64_t>(n - 1, 0);
  const int64_t nf = std::max<int64_t>((n - 1) * (n - 2) / 2, 0);
  const int64_t nc = m.dim == 2 ? nf : std::max<int64_t>((n - 1) * (n - 2) * (n - 3) / 6, 0);
  return m.n_verts + m.n_edges * ne + (m.dim == 3 ? m.n_faces * nf : 0) + m.n_cells * nc;
}

std::string build_topology(Mesh& m) {
  const int d = m.dim;
  const int nv = d + 1;
  // geometry check: no degenerate cell
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * nv];
    for (int i = 0; i < nv; ++i) {
      if (cv[i] < 0 || cv[i] >= m.n_verts) return "cell vertex id out of range";
      for (int j = 0; j < i; ++j)
        if (cv[i] == cv[j]) return "cell with repeated vertex";
    }
    double vol;
    if (d == 2) {
      const double* p0 = &m.coords[cv[0] * 2];
      const double* p1 = &m.coords[cv[1] * 2];
      const double* p2 = &m.coords[cv[2] * 2];
      vol = (p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]);
    } else {
      double J[3][3];
      for (int c2 = 0; c2 < 3; ++c2)
        for (int r = 0; r < 3; ++r) J[r][c2] = m.coords[cv[c2 + 1] * 3 + r] - m.coords[cv[0] * 3 + r];
      vol = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
            J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    }
    if (!(std::fabs(vol) > 0.0) || !std::isfinite(vol)) return "degenerate (zero-volume) cell";
  }
  // unique edges and faces
  std::map<std::pair<int64_t, int64_t>, int64_t> emap;
  std::map<std::array<int64_t, 3>, int64_t> fmap;
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * nv];
    for (int i = 0; i < nv; ++i)
      for (int j = i + 1; j < nv; ++j) emap[{std::min(cv[i], cv[j]), std::max(cv[i], cv[j])}] = 0;
    if (d == 3)
      for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
          for (int k = j + 1; k < 4; ++k) {
            std::array<int64_t, 3> t = {cv[i], cv[j], cv[k]};
            std::sort(t.begin(), t.end());
            fmap[t] = 0;
          }
  }
  m.edges.clear();
  int64_t idx = 0;
  for (auto& kv : emap) {
    kv.second = idx++;
    m.edges.push_back(kv.first.first);
    m.edges.push_back(kv.first.second);
  }
  m.n_edges = idx;
  m.faces.clear();
  idx = 0;
  for (auto& kv : fmap) {
    kv.second = idx++;
    for (int i = 0; i < 3; ++i) m.faces.push_back(kv.first[i]);
  }
  m.n_faces = idx;

  // incidences, ascending cell id
  std::vector<std::vector<Inc>> vinc(m.n_verts), einc(m.n_edges), finc(m.n_faces);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * nv];
    auto corner_of = [&](int64_t v) {
      for (int i = 0; i < nv; ++i)
        if (cv[i] == v) return i;
      return -1;
    };
    for (int i = 0; i < nv; ++i) vinc[cv[i]].push_back(Inc{int(c), {i, -1, -1}});
    for (int i = 0; i < nv; ++i)
      for (int j = i + 1; j < nv; ++j) {
        const int64_t lo = std::min(cv[i], cv[j]), hi = std::max(cv[i], cv[j]);
        einc[emap[{lo, hi}]].push_back(Inc{int(c), {corner_of(lo), corner_of(hi), -1}});
      }
    if (d == 3)
      for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
          for (int k = j + 1; k < 4; ++k) {
            std::array<int64_t, 3> t = {cv[i], cv[j], cv[k]};
            std::sort(t.begin(), t.end());
            finc[fmap[t]].push_back(Inc{int(c), {corner_of(t[0]), corner_of(t[1]), corner_of(t[2])}});
          }
  }
  // conformity and the domain boundary: a facet (edge in 2D, face in 3D)
  // belongs to one cell (boundary) or two (interior)
  m.vertex_bnd.assign(m.n_verts, 0);
  m.edge_bnd.assign(m.n_edges, 0);
  m.face_bnd.assign(m.n_faces, 0);
  if (d == 2) {
    for (int64_t e = 0; e < m.n_edges; ++e) {
      const size_t k = einc[e].size();
      if (k < 1 || k > 2) return "non-conforming mesh: an edge is shared by more than two triangles";
      if (k == 1 && m.bc == 1) {
        m.edge_bnd[e] = 1;
        m.vertex_bnd[m.edges[2 * e]] = 1;
        m.vertex_bnd[m.edges[2 * e + 1]] = 1;
      }
    }
  } else {
    std::map<std::pair<int64_t, int64_t>, int64_t>& em = emap;
    for (int64_t f = 0; f < m.n_faces; ++f) {
      const size_t k = finc[f].size();
      if (k < 1 || k > 2) return "non-conforming mesh: a face is shared by more than two tetrahedra";
      if (k == 1 && m.bc == 1) {
        m.face_bnd[f] = 1;
        const int64_t* fv = &m.faces[3 * f];
        for (int i = 0; i < 3; ++i) m.vertex_bnd[fv[i]] = 1;
        for (int i = 0; i < 3; ++i)
          for (int j = i + 1; j < 3; ++j) m.edge_bnd[em[{fv[i], fv[j]}]] = 1;
      }
    }
  }
  // interface primitives
  m.prims.clear();
  m.incs.clear();
  auto add = [&](int type, int bnd, const std::vector<Inc>& inc) {
    Prim p{type, bnd, int(m.incs.size()), int(inc.size())};
    m.prims.push_back(p);
    m.incs.insert(m.incs.end(), inc.begin(), inc.end());
  };
  for (int64_t v = 0; v < m.n_verts; ++v) {
    if (vinc[v].empty()) return "coarse vertex not used by any cell";
    add(0, m.vertex_bnd[v], vinc[v]);
  }
  for (int64_t e = 0; e < m.n_edges; ++e) add(1, m.edge_bnd[e], einc[e]);
  for (int64_t f = 0; f < m.n_faces; ++f) add(2, m.face_bnd[f], finc[f]);
  return "";
}

std::vector<int4> slab_work_list(int n, int64_t n_cells, int chunks) {
  // cuts at z where the cumulative slice point count passes c/chunks of the
  // macro's slots; items ordered by z-range, then macro
  const int64_t S = (int64_t(n) + 1) * (n + 2) * (n + 3) / 6;
  std::vector<int> cuts = {0};
  int64_t acc = 0;
  for (int z = 0; z <= n; ++z) {
    const int64_t M = n + 1 - z;
    acc += M * (M + 1) / 2;
    if (int(cuts.size()) < chunks && acc * chunks >= S * int64_t(cuts.size()) && z < n) cuts.push_back(z + 1);
  }
  cuts.push_back(n + 1);
  std::vector<int4> items;
  for (size_t c = 0; c + 1 < cuts.size(); ++c)
    for (int64_t mm = 0; mm < n_cells; ++mm)
      if (cuts[c] < cuts[c + 1]) items.push_back(make_int4(int(mm), cuts[c], cuts[c + 1], 0));
  return items;
}

void free_level(const Mesh& m, LevelDev& L) {
  dev_free(m, L.st64);
  dev_free(m, L.st32);
  dev_free(m, L.st_hi);
  dev_free(m, L.st_lo);
  dev_free(m, L.tiles);
  dev_free(m, L.tiles32);
  for (int t = 0; t < 4; ++t) dev_free(m, L.tiles_dt[t]);
  dev_free(m, L.items);
  dev_free(m, L.slabs);
  for (int t = 0; t < 4; ++t) dev_free(m, L.slabs_dt[t]);
  dev_free(m, L.r3_tiles);
  dev_free(m, L.if_slots);
  dev_free(m, L.if_item_base);
  dev_free(m, L.if_pairs);
  dev_free(m, L.if_flat_base);
  dev_free(m, L.if_rest);
  dev_free(m, L.p2_st64);
  dev_free(m, L.p2_st32);
  dev_free(m, L.p2_hi);
  dev_free(m, L.p2_lo);
  dev_free(m, L.p2_items);
  dev_free(m, L.p2_tiles);
  L = LevelDev{};
}

std::vector<int4> tile_list_2d(int n, int rows, int width) {
  std::vector<int4> tl;
  for (int x0 = 1; x0 <= n - 2; x0 += width) {
    const int ymax = n - 1 - x0;
    for (int y0 = 1; y0 <= ymax; y0 += rows) tl.push_back(make_int4(x0, y0, std::min(y0 + rows, ymax + 1), 0));
  }
  // rows of neighbouring strips run side by side, so halo rows hit in L2
  std::stable_sort(tl.begin(), tl.end(), [](const int4& p, const int4& q) {
    if (p.y != q.y) return p.y < q.y;
    return p.x < q.x;
  });
  return tl;
}

bool ff_weights_in_range(const std::vector<double>& st, int per_stencil) {
  for (size_t b = 0; b + per_stencil <= st.size(); b += per_stencil) {
    double wmax = 0.0;  // largest weight of one stencil (class or row group)
    for (int k = 0; k < per_stencil; ++k) wmax = std::max(wmax, std::fabs(st[b + k]));
    if (wmax != 0.0 && !(wmax >= std::ldexp(1.0, -20) && wmax <= std::ldexp(1.0, 14))) return false;
  }
  return true;
}

std::string build_level(Mesh& m, int level, LevelDev& L) {
  const int d = m.dim;
  const int nv = d + 1;
  const int n = 1 << level;
  L.level = level;
  L.n = n;
  L.slots_per_macro = slots_per_macro(d, level);
  const int ncls = d == 2 ? NCLS2 : NCLS3;
  const int nw = d == 2 ? NW2 : NW3;

  // ---- class stencils [cell][class][weight] ------------------------------
  std::vector<double> st(size_t(m.n_cells) * ncls * nw, 0.0);
  int kt[6][4][3];
  kuhn_types(kt);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * nv];
    double* W = &st[size_t(c) * ncls * nw];
    if (d == 2) {
      // micro-element geometry: P(q) = (q_x (v1-v0) + q_y (v2-v0)) / n
      double M[2][2];
      for (int r = 0; r < 2; ++r) {
        M[r][0] = (m.coords[cv[1] * 2 + r] - m.coords[cv[0] * 2 + r]) / n;
        M[r][1] = (m.coords[cv[2] * 2 + r] - m.coords[cv[0] * 2 + r]) / n;
      }
      double K[2][3][3];
      for (int t = 0; t < 2; ++t) {
        double P[3][2];
        for (int s = 0; s < 3; ++s)
          for (int r = 0; r < 2; ++r) P[s][r] = M[r][0] * ELEM2[t][s][0] + M[r][1] * ELEM2[t][s][1];
        tri_stiffness(P, K[t]);
      }
      for (int cls = 0; cls < ncls; ++cls)
        for (int t = 0; t < 2; ++t)
          for (int r = 0; r < 3; ++r) {  // the point is vertex r of the element
            bool ok = true;
            for (int s = 0; s < 3; ++s)
              ok = ok && inside2(cls, ELEM2[t][s][0] - ELEM2[t][r][0], ELEM2[t][s][1] - ELEM2[t][r][1]);
            if (!ok) continue;
            for (int s = 0; s < 3; ++s) {
              const int k = find_off2(ELEM2[t][s][0] - ELEM2[t][r][0], ELEM2[t][s][1] - ELEM2[t][r][1]);
              W[cls * nw + k] += K[t][r][s];
            }
          }
    } else {
      double M[3][3];
      for (int r = 0; r < 3; ++r)
        for (int j = 0; j < 3; ++j) M[r][j] = (m.coords[cv[j + 1] * 3 + r] - m.coords[cv[0] * 3 + r]) / n;
      double K[6][4][4];
      for (int t = 0; t < 6; ++t) {
        double P[4][3];
        for (int s = 0; s < 4; ++s)
          for (int r = 0; r < 3; ++r)
            P[s][r] = M[r][0] * kt[t][s][0] + M[r][1] * kt[t][s][1] + M[r][2] * kt[t][s][2];
        tet_stiffness(P, K[t]);
      }
      for (int cls = 0; cls < ncls; ++cls)
        for (int t = 0; t < 6; ++t)
          for (int r = 0; r < 4; ++r) {
            bool ok = true;
            for (int s = 0; s < 4; ++s)
              ok = ok && inside3(cls, kt[t][s][0] - kt[t][r][0], kt[t][s][1] - kt[t][r][1], kt[t][s][2] - kt[t][r][2]);
            if (!ok) continue;
            for (int s = 0; s < 4; ++s) {
              const int k = find_off3(kt[t][s][0] - kt[t][r][0], kt[t][s][1] - kt[t][r][1], kt[t][s][2] - kt[t][r][2]);
              if (k < 0) return "internal: Kuhn edge outside the 15-point stencil";
              W[cls * nw + k] += K[t][r][s];
            }
          }
    }
  }
  // The operator is symmetric with constant coefficients inside a macro, so
  // the interior stencil satisfies w(d) = w(-d); the sums above give equal
  // values up to rounding.  Make them bitwise equal, so kernels may add
  // opposite neighbours before multiplying.
  for (int64_t c = 0; c < m.n_cells; ++c) {
    double* W = &st[size_t(c) * ncls * nw];
    if (d == 2) {
      const int pairs[3][2] = {{0, 6}, {1, 5}, {2, 4}};  // S/N, SE/NW, W/E
      for (auto& pr : pairs) W[pr[0]] = W[pr[1]] = 0.5 * (W[pr[0]] + W[pr[1]]);
    } else {
      const int pairs[7][2] = {{1, 2}, {3, 4}, {5, 6}, {7, 11}, {8, 12}, {9, 13}, {10, 14}};
      for (auto& pr : pairs) W[pr[0]] = W[pr[1]] = 0.5 * (W[pr[0]] + W[pr[1]]);
    }
  }
  // A weight that vanishes in exact arithmetic (the diagonal couplings of an
  // unjittered Kuhn cube, a right angle in 2D) leaves a rounding residue of a
  // few ulps of the macro's largest weight in the element sums above; such
  // residues (below 2^-46 of the macro's largest weight) are set to zero.
  for (int64_t c = 0; c < m.n_cells; ++c) {
    double* W = &st[size_t(c) * ncls * nw];
    double wmax = 0.0;
    for (int i = 0; i < ncls * nw; ++i) wmax = std::max(wmax, std::fabs(W[i]));
    for (int i = 0; i < ncls * nw; ++i)
      if (std::fabs(W[i]) < std::ldexp(wmax, -46)) W[i] = 0.0;
  }
  L.st_host = st;
  std::vector<float> st32(st.size()), sth(st.size()), stl(st.size());
  for (size_t i = 0; i < st.size(); ++i) {  // float-float parts of 2^40 w (arith.cuh)
    const double ws = std::ldexp(st[i], 40);
    st32[i] = float(st[i]);
    sth[i] = float(ws);
    stl[i] = float(ws - double(sth[i]));
  }
  L.ff_ok = ff_weights_in_range(st, ncls * nw);

  // ---- 2D macro-interior work lists: strips of columns x chunks of rows ----
  // a warp loads 64 consecutive columns and writes the 62 inner ones.  A warp
  // walks its rows one after another, so a level with few tiles would run
  // few long serial walks: the row chunk shrinks from its maximum (8 rows at
  // least) until the level has 16 warps per SM, which keeps small applies
  // and the multigrid's coarse sweeps short.  Maximum chunk: 64 rows for the
  // float64 kernels, 16 for fp32 (measured at level 11, 32 macros: float-
  // float flat within 1 % from 16 to 64 rows, fp32 0.117 ms at 64 rows, 0.109
  // at 16 — more, shorter walks balance its 40 resident warps per SM better).
  int sms = 0;
  if (d == 2 &&
      (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m.device >= 0 ? m.device : 0) != cudaSuccess ||
       sms <= 0)) {
    cudaGetLastError();
    sms = 152;
  }
  auto strips = [&](int th_max, int width) {
    std::vector<int4> tl;
    if (d != 2) return tl;
    auto n_warps = [&](int th) {
      int64_t w = 0;
      for (int x0 = 1; x0 <= n - 2; x0 += width) w += (n - 1 - x0 + th - 1) / th;
      return w * m.n_cells;
    };
    int th = th_max;
    while (th > 8 && n_warps(th) < 16 * int64_t(sms)) th /= 2;
    return tile_list_2d(n, th, width);
  };
  std::vector<int4> tiles = strips(64, kTileWidth2), tiles32 = strips(16, kTileWidth2);
  L.n_tiles32 = int(tiles32.size());
  L.n_tiles = int(tiles.size());

  // ---- interface work list: (prim, b, a0, a1), at most 128 points each ----
  constexpr int IB = 128;
  std::vector<int4> items;
  for (size_t p = 0; p < m.prims.size(); ++p) {
    const Prim& pr = m.prims[p];
    if (pr.type == 0) {
      items.push_back(make_int4(int(p), 0, 0, 1));
    } else if (pr.type == 1) {
      for (int a0 = 1; a0 <= n - 1; a0 += IB) items.push_back(make_int4(int(p), 0, a0, std::min(a0 + IB, n)));
    } else {
      for (int b = 1; b <= n - 2; ++b)
        for (int a0 = 1; a0 <= n - 1 - b; a0 += IB)
          items.push_back(make_int4(int(p), b, a0, std::min(a0 + IB, n - b)));
    }
  }
  L.n_items = int(items.size());

  // ---- 3D slab work list: every macro cut into two z-ranges of about equal
  // point counts (n <= 64, where three slices fit in shared memory); the
  // autotuner may replace it per element type after refinement -------------
  std::vector<int4> slabs;
  if (d == 3 && n <= 64) slabs = slab_work_list(n, m.n_cells, 2);
  L.n_slabs = int(slabs.size());

  std::string err;
  if (!(err = upload(m, &L.st64, st)).empty()) return err;
  if (!(err = upload(m, &L.st32, st32)).empty()) return err;
  if (!(err = upload(m, &L.st_hi, sth)).empty()) return err;
  if (!(err = upload(m, &L.st_lo, stl)).empty()) return err;
  if (!(err = upload(m, &L.tiles, tiles)).empty()) return err;
  if (!(err = upload(m, &L.tiles32, tiles32)).empty()) return err;
  if (!(err = upload(m, &L.items, items)).empty()) return err;
  if (!(err = upload(m, &L.slabs, slabs)).empty()) return err;
  if (d == 3 && !items.empty()) {
    // the slot table of the interface reduction (built on the device)
    std::vector<int64_t> base(items.size() + 1, 0);
    for (size_t i = 0; i < items.size(); ++i)
      base[i + 1] = base[i] + int64_t(items[i].w - items[i].z) * m.prims[items[i].x].inc_count;
    L.n_if_slots = base.back();
    if (!(err = upload(m, &L.if_item_base, base)).empty()) return err;
    std::vector<int64_t> fbase(items.size(), -1);
    std::vector<int> rest;
    int64_t nflat = 0;
    for (size_t i = 0; i < items.size(); ++i) {
      const Prim& pr = m.prims[items[i].x];
      if ((!pr.boundary && pr.inc_count == 2) || (pr.boundary && pr.inc_count == 1)) {
        fbase[i] = nflat;
        nflat += items[i].w - items[i].z;
      } else if (pr.boundary || pr.inc_count > 1) {
        rest.push_back(int(i));
      }
    }
    L.n_if_pairs = nflat;
    L.n_if_rest = int(rest.size());
    if (!(err = upload(m, &L.if_flat_base, fbase)).empty()) return err;
    if (!(err = upload(m, &L.if_rest, rest)).empty()) return err;
    if (nflat > 0) {
      const cudaError_t ep = dev_alloc(m, (void**)&L.if_pairs, size_t(nflat) * sizeof(longlong2));
      if (ep != cudaSuccess) {
        L.if_pairs = nullptr;
        return "device allocation: interface pair table";
      }
    }
    const cudaError_t e = dev_alloc(m, (void**)&L.if_slots, size_t(L.n_if_slots) * sizeof(int64_t));
    if (e != cudaSuccess) {
      L.if_slots = nullptr;
      return "device allocation: interface slot table";
    }
    const cudaError_t e2 = build_iface_slots(m, L, m.mem.stream);
    if (e2 != cudaSuccess) return std::string("cuda: ") + cudaGetErrorString(e2);
  }
  if (d == 3) {
    // row-kernel tiles: every slice z, strips of 30 columns, chunks of 32 rows
    // (level 7, 384 macro-tets: 3.94 -> 3.50 ms float-float and 1.16 -> 1.11
    // ms fp32 against 64-row chunks; a warp walks its rows serially)
    constexpr int R3TH = 32;
    std::vector<int4> r3;
    for (int z = 0; z <= n; ++z) {
      const int M = n + 1 - z;
      for (int x0 = 0; x0 <= M - 1; x0 += 30)
        for (int y0 = 0; y0 <= M - 1 - x0; y0 += R3TH)
          r3.push_back(make_int4(x0, y0, std::min(y0 + R3TH, M - x0), z));
    }
    L.n_r3_tiles = int(r3.size());
    if (!(err = upload(m, &L.r3_tiles, r3)).empty()) return err;
  }
  if (d == 2) return build_p2_level(m, level, L);
  return "";
}

void compute_dof_map(const Mesh& m, int level, int64_t* gid) {
  const int d = m.dim;
  const int nv = d + 1;
  const int64_t n = int64_t(1) << level;
  const int64_t ne = std::max<int64_t>(n - 1, 0);
  const int64_t nf = std::max<int64_t>((n - 1) * (n - 2) / 2, 0);
  const int64_t nc = d == 2 ? nf : std::max<int64_t>((n - 1) * (n - 2) * (n - 3) / 6, 0);
  const int64_t base_e = m.n_verts;
  const int64_t base_f = base_e + m.n_edges * ne;
  const int64_t base_c = base_f + (d == 3 ? m.n_faces * nf : 0);
  const int64_t S = slots_per_macro(d, level);

  std::map<std::pair<int64_t, int64_t>, int64_t> emap;
  for (int64_t e = 0; e < m.n_edges; ++e) emap[{m.edges[2 * e], m.edges[2 * e + 1]}] = e;
  std::map<std::array<int64_t, 3>, int64_t> fmap;
  for (int64_t f = 0; f < m.n_faces; ++f) fmap[{m.faces[3 * f], m.faces[3 * f + 1], m.faces[3 * f + 2]}] = f;

  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * nv];
    int64_t* out = gid + c * S;
    int64_t slot = 0, rank = 0;
    auto classify = [&](const int64_t w[4]) -> int64_t {
      int idx[4], k = 0;
      for (int i = 0; i < nv; ++i)
        if (w[i] > 0) idx[k++] = i;
      if (k == 1) return cv[idx[0]];
      if (k == 2) {
        const int64_t a = cv[idx[0]], b = cv[idx[1]];
        const int64_t lo = std::min(a, b), hi = std::max(a, b);
        const int64_t khi = (a == hi) ? w[idx[0]] : w[idx[1]];
        return base_e + emap.at({lo, hi}) * ne + khi - 1;
      }
      if (k == 3 && d == 3) {
        std::array<std::pair<int64_t, int64_t>, 3> g = {{{cv[idx[0]], w[idx[0]]}, {cv[idx[1]], w[idx[1]]},
                                                        {cv[idx[2]], w[idx[2]]}}};
        std::sort(g.begin(), g.end());
        const int64_t f = fmap.at({g[0].first, g[1].first, g[2].first});
        const int64_t a = g[1].second, b = g[2].second;
        return base_f + f * nf + (b - 1) * (n - 1) - ((b - 1) * b) / 2 + (a - 1);
      }
      return base_c + c * nc + (rank++);
    };
    if (d == 2) {
      for (int64_t y = 0; y <= n; ++y)
        for (int64_t x = 0; x <= n - y; ++x) {
          const int64_t w[4] = {n - x - y, x, y, 0};
          out[slot++] = classify(w);
        }
    } else {
      for (int64_t z = 0; z <= n; ++z)
        for (int64_t y = 0; y <= n - z; ++y)
          for (int64_t x = 0; x <= n - z - y; ++x) {
            const int64_t w[4] = {n - x - y - z, x, y, z};
            out[slot++] = classify(w);
          }
    }
  }
}

}  // namespace hyteg
