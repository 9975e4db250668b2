// Host set-up of the P2 (vertex + edge DoF) operator of a 2D mesh: per-macro
// class stencils from quadratic element matrices, the interface work list of
// the edge DoFs on coarse edges, and the global P2 numbering.
//
// The paper's kernels belong to this discretisation (Sec. 3.1: a vertex array
// and three edge arrays X, Y, XY per macro; Sec. 5.2-5.5: vertex-to-vertex,
// edge-to-vertex, vertex-to-edge and edge-to-edge couplings).  Inside a macro
// all up-triangles are translates of each other and all down-triangles are
// their point reflections, and the P2 stiffness of a triangle does not change
// under scaling, so one element matrix per triangle kind gives every stencil.
//
// Layout per macro: vertex array (the P1 layout), then the X, Y and XY edge
// arrays; edge (x, y) of a group, x + y <= n-1, at y n - y(y-1)/2 + x.
// X(x,y) joins lattice points (x,y)-(x+1,y), Y(x,y) joins (x,y)-(x,y+1),
// XY(x,y) joins (x+1,y)-(x,y+1).
#include <algorithm>
#include <cmath>
#include <map>

#include "hyteg_internal.h"

namespace hyteg {

namespace {

// DoF kinds
enum { KV = 0, KX = 1, KY = 2, KD = 3 };

struct Nb {
  int kind, dx, dy;
};

// Neighbour lists of the four row kinds, in the order of the stencil weights
// (the device kernel uses the same order).
const Nb NBV[P2_NV] = {{KV, 0, 0},  {KV, 1, 0},  {KV, -1, 0}, {KV, 0, 1},  {KV, 0, -1}, {KV, 1, -1}, {KV, -1, 1},
                       {KX, 0, 0},  {KX, -1, 0}, {KX, 0, -1}, {KX, -1, 1}, {KY, 0, 0},  {KY, 0, -1}, {KY, -1, 0},
                       {KY, 1, -1}, {KD, 0, 0},  {KD, -1, 0}, {KD, 0, -1}, {KD, -1, -1}};
const Nb NBX[P2_NE] = {{KV, 0, 0}, {KV, 1, 0}, {KV, 0, 1}, {KV, 1, -1}, {KX, 0, 0},
                       {KY, 0, 0}, {KY, 1, -1}, {KD, 0, 0}, {KD, 0, -1}};
const Nb NBY[P2_NE] = {{KV, 0, 0}, {KV, 0, 1}, {KV, 1, 0}, {KV, -1, 1}, {KY, 0, 0},
                       {KX, 0, 0}, {KX, -1, 1}, {KD, 0, 0}, {KD, -1, 0}};
const Nb NBD[P2_NE] = {{KV, 1, 0}, {KV, 0, 1}, {KV, 0, 0}, {KV, 1, 1}, {KD, 0, 0},
                       {KX, 0, 0}, {KX, 0, 1}, {KY, 0, 0}, {KY, 1, 0}};

// P2 stiffness of the triangle P[0..2]: DoF order v0, v1, v2, e01, e12, e02.
// Basis: lambda_i (2 lambda_i - 1) and 4 lambda_i lambda_j; gradients
// (4 lambda_i - 1) g_i and 4 (lambda_j g_i + lambda_i g_j); integrated with
// the edge-midpoint rule (weights |T|/3), exact for the quadratic integrand.
void p2_tri_stiffness(const double P[3][2], double K[6][6]) {
  const double ax = P[1][0] - P[0][0], ay = P[1][1] - P[0][1];
  const double bx = P[2][0] - P[0][0], by = P[2][1] - P[0][1];
  const double det = ax * by - ay * bx;
  const double area = 0.5 * std::fabs(det);
  // gradients of lambda_1, lambda_2 (rows of J^{-1}), lambda_0 = -(sum)
  double g[3][2];
  g[1][0] = by / det;
  g[1][1] = -bx / det;
  g[2][0] = -ay / det;
  g[2][1] = ax / det;
  g[0][0] = -(g[1][0] + g[2][0]);
  g[0][1] = -(g[1][1] + g[2][1]);
  const int node[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
  const double qp[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) K[a][b] = 0.0;
  for (int q = 0; q < 3; ++q) {
    double gr[6][2];
    for (int a = 0; a < 6; ++a) {
      const int i = node[a][0], j = node[a][1];
      for (int r = 0; r < 2; ++r)
        gr[a][r] = i == j ? (4.0 * qp[q][i] - 1.0) * g[i][r] : 4.0 * (qp[q][j] * g[i][r] + qp[q][i] * g[j][r]);
    }
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) K[a][b] += area / 3.0 * (gr[a][0] * gr[b][0] + gr[a][1] * gr[b][1]);
  }
}

struct Dof {
  int kind, x, y;
};

// The six DoFs of the up-triangle and the down-triangle anchored at (x, y),
// in element order [v0, v1, v2, e01, e12, e02].
void up_dofs(int x, int y, Dof o[6]) {
  o[0] = {KV, x, y};
  o[1] = {KV, x + 1, y};
  o[2] = {KV, x, y + 1};
  o[3] = {KX, x, y};
  o[4] = {KD, x, y};
  o[5] = {KY, x, y};
}
void down_dofs(int x, int y, Dof o[6]) {
  o[0] = {KV, x + 1, y};
  o[1] = {KV, x, y + 1};
  o[2] = {KV, x + 1, y + 1};
  o[3] = {KD, x, y};
  o[4] = {KX, x, y + 1};
  o[5] = {KY, x + 1, y};
}

// Stencil of the DoF `t` of a macro with nt intervals per edge: sum over the
// macro's micro-triangles containing it of the element-matrix rows, each
// coupling placed at its neighbour's slot in `nb`.
std::string accumulate(const Dof& t, int nt, const double Ku[6][6], const double Kd[6][6], const Nb* nb, int nnb,
                       double* W) {
  for (int k = 0; k < nnb; ++k) W[k] = 0.0;
  for (int tri = 0; tri < 2; ++tri)
    for (int y = 0; y < nt; ++y)
      for (int x = 0; x + y <= nt - (tri == 0 ? 1 : 2); ++x) {
        Dof e[6];
        if (tri == 0)
          up_dofs(x, y, e);
        else
          down_dofs(x, y, e);
        for (int a = 0; a < 6; ++a) {
          if (e[a].kind != t.kind || e[a].x != t.x || e[a].y != t.y) continue;
          for (int b = 0; b < 6; ++b) {
            int k = 0;
            while (k < nnb && !(nb[k].kind == e[b].kind && nb[k].dx == e[b].x - t.x && nb[k].dy == e[b].y - t.y)) ++k;
            if (k == nnb) return "internal: P2 coupling outside the stencil";
            W[k] += (tri == 0 ? Ku : Kd)[a][b];
          }
        }
      }
  return "";
}

template <class T>
std::string upload(const Mesh& m, T** d, const std::vector<T>& h) {
  if (h.empty()) {
    *d = nullptr;
    return "";
  }
  if (dev_alloc(m, (void**)d, h.size() * sizeof(T)) != cudaSuccess) {
    *d = nullptr;
    return "device allocation failed";
  }
  const cudaError_t e = dev_upload(m, *d, h.data(), h.size() * sizeof(T));
  return e == cudaSuccess ? "" : std::string("host-to-device copy: ") + cudaGetErrorString(e);
}

}  // namespace

int64_t p2_edge_slots(int level) {
  const int64_t n = int64_t(1) << level;
  return n * (n + 1) / 2;
}

int64_t p2_slots_per_macro(int level) { return slots_per_macro(2, level) + 3 * p2_edge_slots(level); }

std::string build_p2_level(Mesh& m, int level, LevelDev& L) {
  const int n = 1 << level;
  // class stencils at representative DoFs of a macro with 4 intervals per edge
  // (every class has points there; the weights do not depend on the level)
  constexpr int NT = 4;
  const Dof vrep[8] = {{KV, 1, 1}, {KV, 0, 2}, {KV, 2, 0}, {KV, 0, 0}, {KV, 2, 2}, {KV, 0, 4}, {KV, 4, 0}, {KV, 1, 1}};
  const Dof erep[3][2] = {{{KX, 1, 1}, {KX, 1, 0}}, {{KY, 1, 1}, {KY, 0, 1}}, {{KD, 1, 1}, {KD, 1, 2}}};
  const Nb* enb[3] = {NBX, NBY, NBD};
  std::vector<double> st(size_t(m.n_cells) * P2W, 0.0);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * 3];
    double Pu[3][2], Pd[3][2];
    for (int r = 0; r < 2; ++r) {
      const double v0 = m.coords[cv[0] * 2 + r], v1 = m.coords[cv[1] * 2 + r], v2 = m.coords[cv[2] * 2 + r];
      Pu[0][r] = v0;
      Pu[1][r] = v1;
      Pu[2][r] = v2;
      Pd[0][r] = v1;
      Pd[1][r] = v2;
      Pd[2][r] = v1 + v2 - v0;
    }
    double Ku[6][6], Kd[6][6];
    p2_tri_stiffness(Pu, Ku);
    p2_tri_stiffness(Pd, Kd);
    double* W = &st[size_t(c) * P2W];
    std::string err;
    for (int cls = 0; cls < 7; ++cls)
      if (!(err = accumulate(vrep[cls], NT, Ku, Kd, NBV, P2_NV, W + cls * P2_NV)).empty()) return err;
    for (int g = 0; g < 3; ++g)
      for (int cls = 0; cls < 2; ++cls)
        if (!(err = accumulate(erep[g][cls], NT, Ku, Kd, enb[g], P2_NE, W + P2_EOFF + (g * 2 + cls) * P2_NE))
                 .empty())
          return err;
  }
  // For the Laplacian a vertex does not couple with the edge opposite to it in
  // a triangle (integral of (4 lambda_i - 1) lambda_k over T is 4|T|/12 - |T|/3
  // = 0); the quadrature leaves rounding-sized values there.  Store exact
  // zeros: in vertex rows the edges X(-1,1), X(0,-1), Y(-1,0), Y(1,-1),
  // XY(0,0), XY(-1,-1); in edge rows the two vertices off the edge.
  {
    const int vz[6] = {9, 10, 13, 14, 15, 18};
    const int ez[2] = {2, 3};
    for (int64_t c = 0; c < m.n_cells; ++c) {
      double* W = &st[size_t(c) * P2W];
      for (int cls = 0; cls < 8; ++cls)
        for (int k : vz) W[cls * P2_NV + k] = 0.0;
      for (int g = 0; g < 6; ++g)
        for (int k : ez) W[P2_EOFF + g * P2_NE + k] = 0.0;
    }
  }
  std::vector<float> st32(st.size()), sth(st.size()), stl(st.size());
  for (size_t i = 0; i < st.size(); ++i) {  // float-float parts of 2^40 w (arith.cuh)
    const double ws = std::ldexp(st[i], 40);
    st32[i] = float(st[i]);
    sth[i] = float(ws);
    stl[i] = float(ws - double(sth[i]));
  }
  // the largest weight of every vertex class (19) and edge class (9) row
  L.p2_ff_ok = true;
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const std::vector<double> v(st.begin() + c * P2W, st.begin() + c * P2W + P2_EOFF);
    const std::vector<double> e(st.begin() + c * P2W + P2_EOFF, st.begin() + (c + 1) * P2W);
    L.p2_ff_ok = L.p2_ff_ok && ff_weights_in_range(v, P2_NV) && ff_weights_in_range(e, P2_NE);
  }
  // edge DoFs on coarse edges: chunks of at most 128 micro-edges
  std::vector<int4> items;
  for (size_t p = 0; p < m.prims.size(); ++p)
    if (m.prims[p].type == 1)
      for (int t0 = 0; t0 < n; t0 += 128) items.push_back(make_int4(int(p), t0, std::min(t0 + 128, n), 0));
  L.n_p2_items = int(items.size());
  // row-kernel tiles: 30 lattice columns x 16 rows; a DoF of column x has an
  // interior class only on rows y <= n-1-x.  A warp walks its rows serially:
  // at level 10 (32 macros) 16-row chunks beat 64-row ones by 3 % (float-
  // float) and 7 % (fp32), more, shorter walks balancing the SMs better.
  constexpr int TH = 16;
  std::vector<int4> tiles;
  for (int x0 = 0; x0 <= n - 1; x0 += 30) {
    const int ymax = n - 1 - x0;
    for (int y0 = 0; y0 <= ymax; y0 += TH) tiles.push_back(make_int4(x0, y0, std::min(y0 + TH, ymax + 1), 0));
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const int4& a, const int4& b) {
    if (a.y != b.y) return a.y < b.y;
    return a.x < b.x;
  });
  L.n_p2_tiles = int(tiles.size());
  std::string err;
  if (!(err = upload(m, &L.p2_st64, st)).empty()) return err;
  if (!(err = upload(m, &L.p2_st32, st32)).empty()) return err;
  if (!(err = upload(m, &L.p2_hi, sth)).empty()) return err;
  if (!(err = upload(m, &L.p2_lo, stl)).empty()) return err;
  if (!(err = upload(m, &L.p2_items, items)).empty()) return err;
  if (!(err = upload(m, &L.p2_tiles, tiles)).empty()) return err;
  return "";
}

// Global P2 numbering: the P1 numbering of the vertices; then the micro-edges
// on coarse edges (coarse edges in sorted order, n micro-edges each, counted
// from the lower-id end); then the macro-interior micro-edges of every cell in
// cell order and slot order (X with y >= 1, Y with x >= 1, XY with x+y <= n-2).
int64_t p2_n_global(const Mesh& m, int level) {
  const int64_t n = int64_t(1) << level;
  const int64_t inner = 3 * n * (n + 1) / 2 - 3 * n;
  return n_global_dofs(m, level) + m.n_edges * n + m.n_cells * inner;
}

void compute_p2_dof_map(const Mesh& m, int level, int64_t* gid) {
  const int64_t n = int64_t(1) << level;
  const int64_t Sv = slots_per_macro(2, level), Se = p2_edge_slots(level), S2 = Sv + 3 * Se;
  const int64_t base_e = n_global_dofs(m, level);
  const int64_t base_i = base_e + m.n_edges * n;
  const int64_t inner = 3 * n * (n + 1) / 2 - 3 * n;
  std::vector<int64_t> vmap(size_t(Sv * m.n_cells));
  compute_dof_map(m, level, vmap.data());
  std::map<std::pair<int64_t, int64_t>, int64_t> emap;
  for (int64_t e = 0; e < m.n_edges; ++e) emap[{m.edges[2 * e], m.edges[2 * e + 1]}] = e;
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * 3];
    int64_t* out = gid + c * S2;
    for (int64_t s = 0; s < Sv; ++s) out[s] = vmap[size_t(c * Sv + s)];
    // coarse edge of local corners (i, j), i < j: global id of its t-th
    // micro-edge counted from corner i
    auto on_edge = [&](int i, int j, int64_t t) {
      const int64_t a = cv[i], b = cv[j];
      const int64_t e = emap.at({std::min(a, b), std::max(a, b)});
      return base_e + e * n + (a < b ? t : n - 1 - t);
    };
    int64_t rank = 0;
    for (int g = 0; g < 3; ++g) {
      int64_t s = Sv + g * Se;
      for (int64_t y = 0; y < n; ++y)
        for (int64_t x = 0; x + y <= n - 1; ++x, ++s) {
          if (g == 0 && y == 0)
            out[s] = on_edge(0, 1, x);
          else if (g == 1 && x == 0)
            out[s] = on_edge(0, 2, y);
          else if (g == 2 && x + y == n - 1)
            out[s] = on_edge(1, 2, y);  // from corner 1 = (n, 0): y-th micro-edge
          else
            out[s] = base_i + c * inner + (rank++);
        }
    }
  }
}

}  // namespace hyteg
