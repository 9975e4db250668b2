// The Poisson model problem -Laplace u = f, u = 0 on the domain boundary, on
// the refined mesh: its right-hand side in the slot layout, generated on the
// device, and the gather of a slot-layout vector into the global DoF
// numbering.  A solve request of the server is described by a coarse mesh, a
// level and a seed; everything per DoF is made here.
//
// Right-hand side (lumped P1 mass, the load vector of the solver of Sec. 1.2
// with the mass matrix replaced by its row sums):
//   b_i = m_i (f(p_i) + noise * g_i)  off the Dirichlet boundary, 0 on it,
//   m_i = |supp phi_i| / (d+1),  f(p) = prod_k sin(pi p_k),
//   g_i = Box-Muller normal deviate of Philox4x32-10 (Salmon et al., SC'11)
//         with counter (i mod 2^32, i >> 32, 0, 0), key (seed mod 2^32,
//         seed >> 32): u1 = (w0 + 1) 2^-32, u2 = w1 2^-32,
//         g = sqrt(-2 ln u1) cos(2 pi u2),
// where i is the global DoF id (vertices, then edge interiors with edges
// sorted by their vertex ids, then face interiors (3D), then cell interiors).
// p_i is the affine image of the point in its macro for macro-interior
// points and in its interface primitive (from the lowest-id vertex) for the
// others, so all copies of a point are bitwise equal; m_i of an interface
// point sums, over the incident macros in ascending order, the micro-elements
// of that macro containing the point times |macro| / n^d / (d+1).
#include <cmath>
#include <vector>

#include "hyteg_internal.h"

namespace hyteg {

namespace {

constexpr int THREADS = 256;

int grid_for(int64_t n) {
  const int64_t b = (n + THREADS - 1) / THREADS;
  return int(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

__device__ __forceinline__ int64_t slot2(int n, int x, int y) {
  return (int64_t)y * (n + 2) - ((int64_t)y * (y + 1)) / 2 + x;
}
__device__ __forceinline__ int64_t slot3(int n, int x, int y, int z) {
  const int64_t N = n + 1, b = N - z;
  const int64_t zs = N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6;
  return zs + (int64_t)y * b - ((int64_t)y * (y - 1)) / 2 + x;
}
template <int DIM>
__device__ __forceinline__ void unpack(unsigned v, int q[3]) {
  if (DIM == 2) {
    q[0] = int(v & 0xFFFFu);
    q[1] = int(v >> 16);
    q[2] = 0;
  } else {
    q[0] = int(v & 0x7FFu);
    q[1] = int((v >> 11) & 0x7FFu);
    q[2] = int(v >> 22);
  }
}

// Philox4x32-10: ten rounds, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double normal_of(uint64_t id, uint64_t seed) {
  const uint4 w = philox4x32_10(make_uint4(unsigned(id), unsigned(id >> 32), 0u, 0u),
                                make_uint2(unsigned(seed), unsigned(seed >> 32)));
  const double u1 = __dmul_rn((double)w.x + 1.0, 0x1p-32);
  const double u2 = __dmul_rn((double)w.y, 0x1p-32);
  return __dmul_rn(sqrt(__dmul_rn(-2.0, log(u1))), cos(__dmul_rn(2.0 * M_PI, u2)));
}

// b = mass * (prod sin(pi p) + noise * g)
template <int DIM>
__device__ __forceinline__ double rhs_value(const double p[3], double mass, double noise, uint64_t gid,
                                            uint64_t seed) {
  double f = sin(__dmul_rn(M_PI, p[0]));
  for (int r = 1; r < DIM; ++r) f = __dmul_rn(f, sin(__dmul_rn(M_PI, p[r])));
  const double g = noise != 0.0 ? normal_of(gid, seed) : 0.0;
  return __dmul_rn(mass, __dadd_rn(f, __dmul_rn(noise, g)));
}

struct Counts {
  int64_t n_verts, n_edges, n_faces;
  int64_t ne, nf, nc;  // interior points per edge, face, cell
  int64_t base_f, base_c;
};

Counts counts_of(const Mesh& m, int n) {
  Counts k;
  k.n_verts = m.n_verts;
  k.n_edges = m.n_edges;
  k.n_faces = m.n_faces;
  k.ne = n - 1 > 0 ? n - 1 : 0;
  k.nf = n >= 3 ? int64_t(n - 1) * (n - 2) / 2 : 0;
  k.nc = m.dim == 2 ? k.nf : (n >= 4 ? int64_t(n - 1) * (n - 2) * (n - 3) / 6 : 0);
  k.base_f = m.n_verts + m.n_edges * k.ne;
  k.base_c = k.base_f + (m.dim == 3 ? m.n_faces * k.nf : 0);
  return k;
}

// rank of a macro-interior point among the interior points, slot order
template <int DIM>
__device__ __forceinline__ int64_t interior_rank(int n, const int q[3]) {
  const int64_t x = q[0], y = q[1], z = q[2];
  if (DIM == 2) return (y - 1) * (n - 1) - ((y - 1) * y) / 2 + (x - 1);
  auto c3 = [](int64_t k) { return k * (k - 1) * (k - 2) / 6; };
  return c3(n - 1) - c3(n - z) + (y - 1) * (n - 1 - z) - ((y - 1) * y) / 2 + (x - 1);
}

template <int DIM>
__device__ __forceinline__ bool macro_interior(int n, const int q[3]) {
  return DIM == 2 ? (q[0] > 0 && q[1] > 0 && q[0] + q[1] < n)
                  : (q[0] > 0 && q[1] > 0 && q[2] > 0 && q[0] + q[1] + q[2] < n);
}

// Interface point (primitive p, row b, position a): weights on the canonical
// vertices, its global id and its slot in the i-th incident macro.
struct IfacePoint {
  int wv[3];
  int64_t gid;
};

__device__ __forceinline__ IfacePoint iface_point(const Prim& p, int pidx, int a, int b, int n, const Counts& k) {
  IfacePoint r{{0, 0, 0}, 0};
  if (p.type == 0) {
    r.wv[0] = n;
    r.gid = pidx;
  } else if (p.type == 1) {
    r.wv[0] = n - a;
    r.wv[1] = a;
    r.gid = k.n_verts + (pidx - k.n_verts) * k.ne + (a - 1);
  } else {
    r.wv[0] = n - a - b;
    r.wv[1] = a;
    r.wv[2] = b;
    const int64_t f = pidx - k.n_verts - k.n_edges;
    r.gid = k.base_f + f * k.nf + int64_t(b - 1) * (n - 1) - (int64_t(b - 1) * b) / 2 + (a - 1);
  }
  return r;
}

template <int DIM>
__device__ __forceinline__ int64_t copy_slot(const Prim& p, const Inc* __restrict__ incs, int i, const int wv[3],
                                             int n, int64_t S) {
  const Inc inc = incs[p.inc_begin + i];
  int q[3] = {0, 0, 0};
  for (int j = 0; j <= p.type; ++j)
    if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
  return (int64_t)inc.cell * S + (DIM == 2 ? slot2(n, q[0], q[1]) : slot3(n, q[0], q[1], q[2]));
}

template <int DIM>
__global__ void k_rhs_interior(double* __restrict__ b, const unsigned* __restrict__ lpts,
                               const double* __restrict__ cell_x, const double* __restrict__ cell_vol, int n,
                               int64_t S, int64_t total, Counts k, double cnt0, uint64_t seed, double noise) {
  const double inv_n = 1.0 / n;
  const double nd = DIM == 2 ? double(n) * n : double(n) * n * n;
  const SlotDiv divS(S, total);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = divS(i);
    int q[3];
    unpack<DIM>(lpts[i - cell * S], q);
    if (!macro_interior<DIM>(n, q)) continue;
    const double* X = cell_x + cell * 12;
    double p[3];
    for (int r = 0; r < DIM; ++r) {
      double v = X[r];
      for (int j = 1; j <= DIM; ++j)
        v = __dadd_rn(v, __dmul_rn(__dmul_rn(double(q[j - 1]), inv_n), __dsub_rn(X[j * 3 + r], X[r])));
      p[r] = v;
    }
    const double mass = __ddiv_rn(__dmul_rn(cnt0, cell_vol[cell]), __dmul_rn(nd, double(DIM + 1)));
    const int64_t gid = k.base_c + cell * k.nc + interior_rank<DIM>(n, q);
    b[i] = rhs_value<DIM>(p, mass, noise, (uint64_t)gid, seed);
  }
}

template <int DIM>
__global__ void __launch_bounds__(128) k_rhs_iface(double* __restrict__ b, const int4* __restrict__ items,
                                                   const Prim* __restrict__ prims, const Inc* __restrict__ incs,
                                                   const double* __restrict__ prim_x,
                                                   const double* __restrict__ prim_mass, int n, int64_t S, Counts k,
                                                   uint64_t seed, double noise) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  const IfacePoint ip = iface_point(p, it.x, a, it.y, n, k);
  double v = 0.0;
  if (!p.boundary) {
    const double inv_n = 1.0 / n;
    const double nd = DIM == 2 ? double(n) * n : double(n) * n * n;
    const double* X = prim_x + (int64_t)it.x * 9;
    double pt[3];
    for (int r = 0; r < DIM; ++r) {
      double s = X[r];
      for (int j = 1; j <= p.type; ++j)
        s = __dadd_rn(s, __dmul_rn(__dmul_rn(double(ip.wv[j]), inv_n), __dsub_rn(X[j * 3 + r], X[r])));
      pt[r] = s;
    }
    const double mass = __ddiv_rn(prim_mass[it.x], __dmul_rn(nd, double(DIM + 1)));
    v = rhs_value<DIM>(pt, mass, noise, (uint64_t)ip.gid, seed);
  }
  for (int i = 0; i < p.inc_count; ++i) b[copy_slot<DIM>(p, incs, i, ip.wv, n, S)] = v;
}

template <int DIM>
__global__ void k_global_interior(double* __restrict__ out, const double* __restrict__ v,
                                  const unsigned* __restrict__ lpts, int n, int64_t S, int64_t total, Counts k) {
  const SlotDiv divS(S, total);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = divS(i);
    int q[3];
    unpack<DIM>(lpts[i - cell * S], q);
    if (!macro_interior<DIM>(n, q)) continue;
    out[k.base_c + cell * k.nc + interior_rank<DIM>(n, q)] = v[i];
  }
}

// the copy in the lowest-id incident macro is the one gathered
template <int DIM>
__global__ void __launch_bounds__(128) k_global_iface(double* __restrict__ out, const double* __restrict__ v,
                                                      const int4* __restrict__ items, const Prim* __restrict__ prims,
                                                      const Inc* __restrict__ incs, int n, int64_t S, Counts k) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  const IfacePoint ip = iface_point(p, it.x, a, it.y, n, k);
  out[ip.gid] = v[copy_slot<DIM>(p, incs, 0, ip.wv, n, S)];
}

template <class T>
std::string upload(const Mesh& m, T** d, const std::vector<T>& h) {
  if (dev_alloc(m, (void**)d, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) {
    *d = nullptr;
    return "device allocation failed";
  }
  const cudaError_t e = dev_upload(m, *d, h.data(), h.size() * sizeof(T));
  return e == cudaSuccess ? "" : std::string("cuda: ") + cudaGetErrorString(e);
}

}  // namespace

std::string problem_setup(Mesh& m) {
  if (m.problem.ready) return "";
  const int d = m.dim;
  const int64_t nc = m.n_cells;
  std::vector<double> cx(size_t(nc) * 12, 0.0), vol(nc);
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t* cv = &m.cells[c * (d + 1)];
    for (int j = 0; j <= d; ++j)
      for (int r = 0; r < d; ++r) cx[size_t(c) * 12 + j * 3 + r] = m.coords[cv[j] * d + r];
    vol[c] = cell_measure(m, c);
  }
  std::vector<double> px(m.prims.size() * 9, 0.0), pm(m.prims.size(), 0.0);
  for (size_t p = 0; p < m.prims.size(); ++p) {
    const Prim& pr = m.prims[p];
    const Inc& first = m.incs[pr.inc_begin];
    const int64_t* cv0 = &m.cells[int64_t(first.cell) * (d + 1)];
    for (int j = 0; j <= pr.type; ++j)
      for (int r = 0; r < d; ++r) px[p * 9 + j * 3 + r] = m.coords[cv0[first.corner[j]] * d + r];
    double s = 0.0;
    for (int i = 0; i < pr.inc_count; ++i) {
      const Inc& inc = m.incs[pr.inc_begin + i];
      // the class of the primitive's points in this cell: the faces opposite
      // the corners that carry no weight
      bool used[4] = {false, false, false, false};
      for (int j = 0; j <= pr.type; ++j) used[inc.corner[j]] = true;
      int cls = 0;
      if (!used[1]) cls |= 1;
      if (!used[2]) cls |= 2;
      if (d == 2) {
        if (!used[0]) cls |= 4;
      } else {
        if (!used[3]) cls |= 4;
        if (!used[0]) cls |= 8;
      }
      s += double(elements_at_class(d, cls)) * vol[inc.cell];
    }
    pm[p] = s;
  }
  std::string err;
  if (!(err = upload(m, &m.problem.cell_x, cx)).empty()) return err;
  if (!(err = upload(m, &m.problem.cell_vol, vol)).empty()) return err;
  if (!(err = upload(m, &m.problem.prim_x, px)).empty()) return err;
  if (!(err = upload(m, &m.problem.prim_mass, pm)).empty()) return err;
  const cudaError_t e = dev_sync(m);
  if (e != cudaSuccess) return std::string("cuda: ") + cudaGetErrorString(e);
  m.problem.ready = true;
  return "";
}

void problem_free(Mesh& m) {
  dev_free(m, m.problem.cell_x);
  dev_free(m, m.problem.cell_vol);
  dev_free(m, m.problem.prim_x);
  dev_free(m, m.problem.prim_mass);
  m.problem = ProblemDev{};
}

cudaError_t poisson_rhs(const Mesh& m, int level, uint64_t seed, double noise, double* b, cudaStream_t s) {
  const LevelDev& L = m.levels[level];
  const MgLevel& g = m.solver->lv[level];
  const int64_t S = L.slots_per_macro, total = S * m.n_cells;
  const Counts k = counts_of(m, L.n);
  const double cnt0 = elements_at_class(m.dim, 0);
  if (m.dim == 2)
    k_rhs_interior<2><<<grid_for(total), THREADS, 0, s>>>(b, g.lpts, m.problem.cell_x, m.problem.cell_vol, L.n, S,
                                                           total, k, cnt0, seed, noise);
  else
    k_rhs_interior<3><<<grid_for(total), THREADS, 0, s>>>(b, g.lpts, m.problem.cell_x, m.problem.cell_vol, L.n, S,
                                                           total, k, cnt0, seed, noise);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || L.n_items == 0) return e;
  if (m.dim == 2)
    k_rhs_iface<2><<<L.n_items, 128, 0, s>>>(b, L.items, m.d_prims, m.d_incs, m.problem.prim_x, m.problem.prim_mass,
                                              L.n, S, k, seed, noise);
  else
    k_rhs_iface<3><<<L.n_items, 128, 0, s>>>(b, L.items, m.d_prims, m.d_incs, m.problem.prim_x, m.problem.prim_mass,
                                              L.n, S, k, seed, noise);
  return cudaGetLastError();
}

cudaError_t to_global(const Mesh& m, int level, const double* v, double* out, cudaStream_t s) {
  const LevelDev& L = m.levels[level];
  const MgLevel& g = m.solver->lv[level];
  const int64_t S = L.slots_per_macro, total = S * m.n_cells;
  const Counts k = counts_of(m, L.n);
  if (m.dim == 2)
    k_global_interior<2><<<grid_for(total), THREADS, 0, s>>>(out, v, g.lpts, L.n, S, total, k);
  else
    k_global_interior<3><<<grid_for(total), THREADS, 0, s>>>(out, v, g.lpts, L.n, S, total, k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || L.n_items == 0) return e;
  if (m.dim == 2)
    k_global_iface<2><<<L.n_items, 128, 0, s>>>(out, v, L.items, m.d_prims, m.d_incs, L.n, S, k);
  else
    k_global_iface<3><<<L.n_items, 128, 0, s>>>(out, v, L.items, m.d_prims, m.d_incs, L.n, S, k);
  return cudaGetLastError();
}

}  // namespace hyteg
