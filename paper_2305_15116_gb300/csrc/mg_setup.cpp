// Host set-up of the multigrid solver and the geometric queries it needs:
// slot coordinates, lumped masses, per-level inverse diagonals, owner
// weights for norms, multiplicities for the restriction and the inverse of
// the level-0 operator.
//
// The paper uses the refinement levels as the multigrid hierarchy (Sec. 1.2)
// and names smoothers among the generated kernels (Sec. 5.1); the cycle
// itself (weighted Jacobi, linear interpolation, R = P^T) is the textbook one.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>

#include "hyteg_internal.h"

namespace hyteg {

namespace {

struct PointRef {
  int64_t cell;
  int q[3];
};

// Local coordinates of every slot of one macro, in slot order.
std::vector<std::array<int, 3>> local_points(int dim, int n) {
  std::vector<std::array<int, 3>> pts;
  if (dim == 2) {
    for (int y = 0; y <= n; ++y)
      for (int x = 0; x <= n - y; ++x) pts.push_back({x, y, 0});
  } else {
    for (int z = 0; z <= n; ++z)
      for (int y = 0; y <= n - z; ++y)
        for (int x = 0; x <= n - z - y; ++x) pts.push_back({x, y, z});
  }
  return pts;
}

int64_t slot_of(int dim, int n, const int q[3]) {
  if (dim == 2) return (int64_t)q[1] * (n + 2) - ((int64_t)q[1] * (q[1] + 1)) / 2 + q[0];
  const int64_t N = n + 1, b = N - q[2];
  const int64_t zs = N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6;
  return zs + (int64_t)q[1] * b - ((int64_t)q[1] * (q[1] - 1)) / 2 + q[0];
}

int point_class(int dim, int n, const int q[3]) {
  if (dim == 2) return (q[0] == 0 ? 1 : 0) | (q[1] == 0 ? 2 : 0) | (q[0] + q[1] == n ? 4 : 0);
  return (q[0] == 0 ? 1 : 0) | (q[1] == 0 ? 2 : 0) | (q[2] == 0 ? 4 : 0) | (q[0] + q[1] + q[2] == n ? 8 : 0);
}

// Calls f(point index a, b, list of copies) for every point of every
// interface primitive (coarse vertex, edge, face) at level n.
template <class F>
void for_each_interface_point(const Mesh& m, int n, F f) {
  const int d = m.dim;
  std::vector<PointRef> refs;
  for (size_t p = 0; p < m.prims.size(); ++p) {
    const Prim& pr = m.prims[p];
    auto visit = [&](int a, int b) {
      int wv[3] = {0, 0, 0};
      if (pr.type == 0) {
        wv[0] = n;
      } else if (pr.type == 1) {
        wv[0] = n - a;
        wv[1] = a;
      } else {
        wv[0] = n - a - b;
        wv[1] = a;
        wv[2] = b;
      }
      refs.clear();
      for (int i = 0; i < pr.inc_count; ++i) {
        const Inc& inc = m.incs[pr.inc_begin + i];
        PointRef r{inc.cell, {0, 0, 0}};
        for (int j = 0; j <= pr.type; ++j)
          if (inc.corner[j] >= 1) r.q[inc.corner[j] - 1] += wv[j];
        refs.push_back(r);
      }
      f(pr, refs);
    };
    if (pr.type == 0) {
      visit(0, 0);
    } else if (pr.type == 1) {
      for (int a = 1; a <= n - 1; ++a) visit(a, 0);
    } else {
      for (int b = 1; b <= n - 2; ++b)
        for (int a = 1; a <= n - 1 - b; ++a) visit(a, b);
    }
    (void)d;
  }
}

template <class T>
std::string upload_vec(const Mesh& m, T** dptr, const std::vector<T>& h) {
  cudaError_t e = dev_alloc(m, (void**)dptr, std::max<size_t>(h.size(), 1) * sizeof(T));
  if (e != cudaSuccess) {
    *dptr = nullptr;
    return std::string("cuda: device allocation: ") + cudaGetErrorString(e);
  }
  e = dev_upload(m, *dptr, h.data(), h.size() * sizeof(T));
  if (e != cudaSuccess) return std::string("cuda: host-to-device copy: ") + cudaGetErrorString(e);
  return "";
}

template <class T>
std::string alloc_vec(const Mesh& m, T** dptr, size_t count) {
  cudaError_t e = dev_alloc(m, (void**)dptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    *dptr = nullptr;
    return std::string("cuda: device allocation: ") + cudaGetErrorString(e);
  }
  e = dev_zero(m, *dptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return std::string("cuda: clear: ") + cudaGetErrorString(e);
  return "";
}

}  // namespace

double cell_measure(const Mesh& m, int64_t c) {
  const int d = m.dim;
  const int64_t* cv = &m.cells[c * (d + 1)];
  if (d == 2) {
    const double* p0 = &m.coords[cv[0] * 2];
    const double* p1 = &m.coords[cv[1] * 2];
    const double* p2 = &m.coords[cv[2] * 2];
    return 0.5 * std::fabs((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]));
  }
  double J[3][3];
  for (int j = 0; j < 3; ++j)
    for (int r = 0; r < 3; ++r) J[r][j] = m.coords[cv[j + 1] * 3 + r] - m.coords[cv[0] * 3 + r];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  return std::fabs(det) / 6.0;
}

// Number of micro-elements of a macro that contain a point of boundary
// class `cls` (independent of the macro and the level): 6 / 24 inside.
int elements_at_class(int dim, int cls) {
  static const int E2[2][3][2] = {{{0, 0}, {1, 0}, {0, 1}}, {{1, 0}, {0, 1}, {1, 1}}};
  int count = 0;
  if (dim == 2) {
    for (int t = 0; t < 2; ++t)
      for (int r = 0; r < 3; ++r) {
        bool ok = true;
        for (int s = 0; s < 3; ++s) {
          const int dx = E2[t][s][0] - E2[t][r][0], dy = E2[t][s][1] - E2[t][r][1];
          if (((cls & 1) && dx < 0) || ((cls & 2) && dy < 0) || ((cls & 4) && dx + dy > 0)) ok = false;
        }
        count += ok;
      }
    return count;
  }
  int perm[3] = {0, 1, 2};
  do {
    int u[4][3] = {{0, 0, 0}};
    for (int s = 1; s < 4; ++s) {
      for (int c = 0; c < 3; ++c) u[s][c] = u[s - 1][c];
      u[s][perm[s - 1]] += 1;
    }
    int o[4][3];
    for (int s = 0; s < 4; ++s) {
      o[s][0] = u[s][0] - u[s][1];
      o[s][1] = u[s][1] - u[s][2];
      o[s][2] = u[s][2];
    }
    for (int r = 0; r < 4; ++r) {
      bool ok = true;
      for (int s = 0; s < 4; ++s) {
        const int dx = o[s][0] - o[r][0], dy = o[s][1] - o[r][1], dz = o[s][2] - o[r][2];
        if (((cls & 1) && dx < 0) || ((cls & 2) && dy < 0) || ((cls & 4) && dz < 0) ||
            ((cls & 8) && dx + dy + dz > 0))
          ok = false;
      }
      count += ok;
    }
  } while (std::next_permutation(perm, perm + 3));
  return count;
}


void compute_slot_coords(const Mesh& m, int level, double* xyz) {
  // Every copy of an interface point gets the coordinates of the primitive's
  // own parameterisation, so copies are bitwise equal; macro-interior points
  // use the macro's affine map.
  const int d = m.dim;
  const int n = 1 << level;
  const int64_t S = slots_per_macro(d, level);
  const auto pts = local_points(d, n);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * (d + 1)];
    for (int64_t s = 0; s < S; ++s) {
      double* o = xyz + (c * S + s) * d;
      for (int r = 0; r < d; ++r) {
        double v = m.coords[cv[0] * d + r];
        for (int j = 0; j < d; ++j) v += (double(pts[s][j]) / n) * (m.coords[cv[j + 1] * d + r] - m.coords[cv[0] * d + r]);
        o[r] = v;
      }
    }
  }
  for (size_t p = 0; p < m.prims.size(); ++p) {
    const Prim& pr = m.prims[p];
    // canonical vertices of the primitive: sorted global ids
    std::array<int64_t, 3> gv{};
    {
      const Inc& inc = m.incs[pr.inc_begin];
      const int64_t* cv = &m.cells[int64_t(inc.cell) * (d + 1)];
      for (int j = 0; j <= pr.type; ++j) gv[j] = cv[inc.corner[j]];
    }
    auto put = [&](int a, int b) {
      int wv[3] = {0, 0, 0};
      if (pr.type == 0) {
        wv[0] = n;
      } else if (pr.type == 1) {
        wv[0] = n - a;
        wv[1] = a;
      } else {
        wv[0] = n - a - b;
        wv[1] = a;
        wv[2] = b;
      }
      double pos[3] = {0, 0, 0};
      for (int r = 0; r < d; ++r) {
        pos[r] = m.coords[gv[0] * d + r];
        for (int j = 1; j <= pr.type; ++j)
          pos[r] += (double(wv[j]) / n) * (m.coords[gv[j] * d + r] - m.coords[gv[0] * d + r]);
      }
      for (int i = 0; i < pr.inc_count; ++i) {
        const Inc& inc = m.incs[pr.inc_begin + i];
        int q[3] = {0, 0, 0};
        for (int j = 0; j <= pr.type; ++j)
          if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
        double* o = xyz + (int64_t(inc.cell) * S + slot_of(d, n, q)) * d;
        for (int r = 0; r < d; ++r) o[r] = pos[r];
      }
    };
    if (pr.type == 0) {
      put(0, 0);
    } else if (pr.type == 1) {
      for (int a = 1; a <= n - 1; ++a) put(a, 0);
    } else {
      for (int b = 1; b <= n - 2; ++b)
        for (int a = 1; a <= n - 1 - b; ++a) put(a, b);
    }
  }
}

void compute_lumped_mass(const Mesh& m, int level, double* mass) {
  // Lumped P1 mass |supp phi_i| / (d+1): each macro contributes the micro-
  // elements of its own that contain the point (a count that depends only on
  // the point's boundary class) times |macro| / n^d / (d+1); the interface
  // points sum these partials over the incident macros in ascending order.
  const int d = m.dim;
  const int n = 1 << level;
  const int64_t S = slots_per_macro(d, level);
  const int ncls = d == 2 ? NCLS2 : NCLS3;
  std::vector<int> cnt(ncls);
  for (int c = 0; c < ncls; ++c) cnt[c] = elements_at_class(d, c);
  const auto pts = local_points(d, n);
  const double nd = d == 2 ? double(n) * n : double(n) * n * n;
  std::vector<double> unit(m.n_cells);
  for (int64_t c = 0; c < m.n_cells; ++c) unit[c] = cell_measure(m, c) / nd / (d + 1);
  for (int64_t c = 0; c < m.n_cells; ++c)
    for (int64_t s = 0; s < S; ++s) {
      const int q[3] = {pts[s][0], pts[s][1], pts[s][2]};
      mass[c * S + s] = cnt[point_class(d, n, q)] * unit[c];
    }
  for_each_interface_point(m, n, [&](const Prim&, const std::vector<PointRef>& refs) {
    double sum = 0.0;
    for (const auto& r : refs) sum += mass[r.cell * S + slot_of(d, n, r.q)];
    for (const auto& r : refs) mass[r.cell * S + slot_of(d, n, r.q)] = sum;
  });
}

void compute_dirichlet_mask(const Mesh& m, int level, unsigned char* mask) {
  const int d = m.dim;
  const int n = 1 << level;
  const int64_t S = slots_per_macro(d, level);
  std::fill(mask, mask + S * m.n_cells, (unsigned char)0);
  for_each_interface_point(m, n, [&](const Prim& pr, const std::vector<PointRef>& refs) {
    if (!pr.boundary) return;
    for (const auto& r : refs) mask[r.cell * S + slot_of(d, n, r.q)] = 1;
  });
}

void solver_free(Mesh& m) {
  if (!m.solver) return;
  Solver& sv = *m.solver;
  for (cudaGraphExec_t g : sv.graph32)
    if (g) cudaGraphExecDestroy(g);
  for (cudaGraphExec_t g : sv.graph64)
    if (g) cudaGraphExecDestroy(g);
  for (auto& L : sv.lv) {
    dev_free(m, L.dinv64);
    dev_free(m, L.dinv32);
    dev_free(m, L.owner);
    dev_free(m, L.lpts);
    dev_free(m, L.multinv64);
    dev_free(m, L.multinv32);
    dev_free(m, L.u64);
    dev_free(m, L.b64);
    dev_free(m, L.y64);
    dev_free(m, L.r64);
    dev_free(m, L.u32);
    dev_free(m, L.b32);
    dev_free(m, L.y32);
    dev_free(m, L.r32);
  }
  dev_free(m, sv.a0inv64);
  dev_free(m, sv.a0inv32);
  dev_free(m, sv.v_of_slot0);
  dev_free(m, sv.slot_of_v0);
  dev_free(m, sv.red);
  delete m.solver;
  m.solver = nullptr;
}

std::string solver_setup(Mesh& m, int max_level, int nu1, int nu2, double omega) {
  const int d = m.dim;
  const int ncls = d == 2 ? NCLS2 : NCLS3;
  const int nw = d == 2 ? NW2 : NW3;
  if (m.n_verts > 4096) return "the coarsest level has more than 4096 vertices (dense direct solve)";
  solver_free(m);
  if (d == 3) {
    const cudaError_t e = slab3d_prepare();  // before any captured cycle
    if (e != cudaSuccess) return std::string("cuda: ") + cudaGetErrorString(e);
  }
  m.solver = new Solver();
  Solver& sv = *m.solver;
  sv.max_level = max_level;
  sv.nu1 = nu1;
  sv.nu2 = nu2;
  sv.omega = omega;
  std::string err;

  // multiplicity of each macro-boundary class: the number of cells sharing
  // the primitive (vertex, edge, face) that a point of that class lies in
  std::map<std::vector<int64_t>, int> inc_count;
  for (const Prim& pr : m.prims) {
    const Inc& inc = m.incs[pr.inc_begin];
    const int64_t* cv = &m.cells[int64_t(inc.cell) * (d + 1)];
    std::vector<int64_t> key;
    for (int j = 0; j <= pr.type; ++j) key.push_back(cv[inc.corner[j]]);
    std::sort(key.begin(), key.end());
    inc_count[key] = pr.inc_count;
  }
  std::vector<double> multinv(size_t(m.n_cells) * ncls, 1.0);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * (d + 1)];
    for (int cls = 1; cls < ncls; ++cls) {
      // corners not opposite an active face: x=0 is opposite corner 1, y=0
      // corner 2, z=0 corner 3 (3D), x+y(+z)=n corner 0
      bool drop[4] = {false, false, false, false};
      if (cls & 1) drop[1] = true;
      if (cls & 2) drop[2] = true;
      if (d == 2) {
        if (cls & 4) drop[0] = true;
      } else {
        if (cls & 4) drop[3] = true;
        if (cls & 8) drop[0] = true;
      }
      std::vector<int64_t> key;
      for (int j = 0; j <= d; ++j)
        if (!drop[j]) key.push_back(cv[j]);
      if (key.empty() || int(key.size()) > d) continue;  // impossible class
      std::sort(key.begin(), key.end());
      auto it = inc_count.find(key);
      if (it != inc_count.end()) multinv[size_t(c) * ncls + cls] = 1.0 / it->second;
    }
  }
  std::vector<float> multinv32(multinv.begin(), multinv.end());

  for (int l = 0; l <= max_level; ++l) {
    const LevelDev& L = m.levels[l];
    const int n = 1 << l;
    const int64_t S = L.slots_per_macro;
    const int64_t ns = S * m.n_cells;
    sv.lv.push_back(MgLevel{});
    MgLevel& g = sv.lv.back();
    g.level = l;
    const auto pts = local_points(d, n);
    std::vector<unsigned> lp(S);
    for (int64_t s = 0; s < S; ++s)
      lp[s] = d == 2 ? unsigned(pts[s][0]) | (unsigned(pts[s][1]) << 16)
                     : unsigned(pts[s][0]) | (unsigned(pts[s][1]) << 11) | (unsigned(pts[s][2]) << 22);
    if (!(err = upload_vec(m, &g.lpts, lp)).empty()) return err;
    if (!(err = upload_vec(m, &g.multinv64, multinv)).empty()) return err;
    if (!(err = upload_vec(m, &g.multinv32, multinv32)).empty()) return err;
    if (!(err = alloc_vec(m, &g.dinv64, ns)).empty()) return err;
    if (!(err = alloc_vec(m, &g.dinv32, ns)).empty()) return err;
    if (!(err = alloc_vec(m, &g.owner, ns)).empty()) return err;
    for (double** v : {&g.u64, &g.b64, &g.y64, &g.r64})
      if (!(err = alloc_vec(m, v, ns)).empty()) return err;
    for (float** v : {&g.u32, &g.b32, &g.y32, &g.r32})
      if (!(err = alloc_vec(m, v, ns)).empty()) return err;
    // inverse diagonals and owner flags on the device: partial diagonals ->
    // interface sums in ascending macro order -> Dirichlet rows -> inverse
    const cudaError_t e = mg_diag_setup(m, l, g, m.mem.stream);
    if (e != cudaSuccess) return std::string("cuda: diagonal set-up: ") + cudaGetErrorString(e);
  }

  // level 0: the coarse operator on the coarse vertices, dense inverse
  const int V = int(m.n_verts);
  sv.nv0 = V;
  const LevelDev& L0 = m.levels[0];
  std::vector<double> A(size_t(V) * V, 0.0);
  std::vector<int> v_of_slot(size_t(m.n_cells) * (d + 1)), slot_of_v(V, -1);
  const int off2[NW2][2] = {{0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}};
  const int off3[NW3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                            {1, -1, 0}, {-1, 1, 0}, {0, 0, 1},  {-1, 0, 1}, {0, -1, 1},
                            {1, -1, 1}, {0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {-1, 1, -1}};
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const int64_t* cv = &m.cells[c * (d + 1)];
    for (int i = 0; i <= d; ++i) {
      // corner i at local point e_i (corner 0 at the origin)
      int q[3] = {0, 0, 0};
      if (i >= 1) q[i - 1] = 1;
      const int64_t sl = c * (d + 1) + slot_of(d, 1, q);
      v_of_slot[sl] = int(cv[i]);
      if (slot_of_v[cv[i]] < 0) slot_of_v[cv[i]] = int(sl);
      const int cls = point_class(d, 1, q);
      for (int k = 0; k < nw; ++k) {
        int t[3] = {q[0], q[1], q[2]};
        if (d == 2) {
          t[0] += off2[k][0];
          t[1] += off2[k][1];
        } else {
          t[0] += off3[k][0];
          t[1] += off3[k][1];
          t[2] += off3[k][2];
        }
        if (t[0] < 0 || t[1] < 0 || t[2] < 0 || t[0] + t[1] + t[2] > 1) continue;
        int j = 0;  // corner at local point t
        for (int r = 0; r < d; ++r)
          if (t[r] == 1) j = r + 1;
        const double w = L0.st_host[(size_t(c) * ncls + cls) * nw + k];
        A[size_t(cv[i]) * V + cv[j]] += w;
      }
    }
  }
  for (int v = 0; v < V; ++v)
    if (m.vertex_bnd[v]) {
      for (int j = 0; j < V; ++j) A[size_t(v) * V + j] = 0.0;
      A[size_t(v) * V + v] = 1.0;
    }
  // Gauss-Jordan inverse with partial pivoting
  std::vector<double> inv(size_t(V) * V, 0.0);
  for (int i = 0; i < V; ++i) inv[size_t(i) * V + i] = 1.0;
  for (int col = 0; col < V; ++col) {
    int piv = col;
    for (int r = col + 1; r < V; ++r)
      if (std::fabs(A[size_t(r) * V + col]) > std::fabs(A[size_t(piv) * V + col])) piv = r;
    if (std::fabs(A[size_t(piv) * V + col]) == 0.0) return "level-0 operator is singular (no Dirichlet boundary?)";
    if (piv != col)
      for (int j = 0; j < V; ++j) {
        std::swap(A[size_t(piv) * V + j], A[size_t(col) * V + j]);
        std::swap(inv[size_t(piv) * V + j], inv[size_t(col) * V + j]);
      }
    const double p = A[size_t(col) * V + col];
    for (int j = 0; j < V; ++j) {
      A[size_t(col) * V + j] /= p;
      inv[size_t(col) * V + j] /= p;
    }
    for (int r = 0; r < V; ++r)
      if (r != col) {
        const double f = A[size_t(r) * V + col];
        if (f == 0.0) continue;
        for (int j = 0; j < V; ++j) {
          A[size_t(r) * V + j] -= f * A[size_t(col) * V + j];
          inv[size_t(r) * V + j] -= f * inv[size_t(col) * V + j];
        }
      }
  }
  std::vector<float> inv32(inv.begin(), inv.end());
  if (!(err = upload_vec(m, &sv.a0inv64, inv)).empty()) return err;
  if (!(err = upload_vec(m, &sv.a0inv32, inv32)).empty()) return err;
  if (!(err = upload_vec(m, &sv.v_of_slot0, v_of_slot)).empty()) return err;
  if (!(err = upload_vec(m, &sv.slot_of_v0, slot_of_v)).empty()) return err;
  if (!(err = alloc_vec(m, &sv.red, size_t(1024 + 8))).empty()) return err;
  const cudaError_t e = dev_sync(m);
  if (e != cudaSuccess) return std::string("cuda: set-up: ") + cudaGetErrorString(e);
  return "";
}

}  // namespace hyteg
