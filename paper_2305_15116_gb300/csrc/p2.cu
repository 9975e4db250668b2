// P2 operator apply (2D): the vertex-to-vertex, edge-to-vertex,
// vertex-to-edge and edge-to-edge kernels of Sec. 4.2-4.5 merged into one
// pass, as the paper proposes for its next step (Sec. 6: one kernel instead
// of four, so every array is read and written once).
//
// One thread per lattice point (x, y) of a macro computes up to four rows:
// the vertex DoF (x, y) (19 couplings: 7 vertices, 4 edges of each group)
// and the edges X(x,y), Y(x,y), XY(x,y) when x + y <= n-1 (9 couplings each:
// 4 vertices, 4 edges and the edge itself).  DoFs inside the macro use the
// macro's full stencils; DoFs on the macro's edges use partial stencils of
// their class (only the macro's own micro-triangles), and a reduction over
// the copies of every interface DoF (ascending macro order) completes them,
// as for P1; Dirichlet DoFs get y = x.
//
// Layout per macro: vertex array (row y at y(n+2) - y(y+1)/2), then the X, Y
// and XY edge arrays, edge (x, y) at y n - y(y-1)/2 + x.
#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

enum { KV = 0, KX = 1, KY = 2, KD = 3 };

struct NbD {
  int kind, dx, dy;
};

// Neighbour order of the stencil weights (p2_setup.cpp builds them in this order).
__constant__ NbD c_nbv[P2_NV] = {{KV, 0, 0},  {KV, 1, 0},  {KV, -1, 0}, {KV, 0, 1},  {KV, 0, -1},
                                  {KV, 1, -1}, {KV, -1, 1}, {KX, 0, 0},  {KX, -1, 0}, {KX, 0, -1},
                                  {KX, -1, 1}, {KY, 0, 0},  {KY, 0, -1}, {KY, -1, 0}, {KY, 1, -1},
                                  {KD, 0, 0},  {KD, -1, 0}, {KD, 0, -1}, {KD, -1, -1}};
__constant__ NbD c_nbe[3][P2_NE] = {
    {{KV, 0, 0}, {KV, 1, 0}, {KV, 0, 1}, {KV, 1, -1}, {KX, 0, 0}, {KY, 0, 0}, {KY, 1, -1}, {KD, 0, 0}, {KD, 0, -1}},
    {{KV, 0, 0}, {KV, 0, 1}, {KV, 1, 0}, {KV, -1, 1}, {KY, 0, 0}, {KX, 0, 0}, {KX, -1, 1}, {KD, 0, 0}, {KD, -1, 0}},
    {{KV, 1, 0}, {KV, 0, 1}, {KV, 0, 0}, {KV, 1, 1}, {KD, 0, 0}, {KX, 0, 0}, {KX, 0, 1}, {KY, 0, 0}, {KY, 1, 0}}};

struct Geo {
  int n;
  int64_t Sv, Se, S2;
  __device__ __forceinline__ int64_t vidx(int x, int y) const {
    return (int64_t)y * (n + 2) - ((int64_t)y * (y + 1)) / 2 + x;
  }
  __device__ __forceinline__ int64_t eidx(int g, int x, int y) const {
    return Sv + g * Se + (int64_t)y * n - ((int64_t)y * (y - 1)) / 2 + x;
  }
  __device__ __forceinline__ int64_t idx(int kind, int x, int y) const {
    return kind == KV ? vidx(x, y) : eidx(kind - 1, x, y);
  }
  __device__ __forceinline__ bool valid(int kind, int x, int y) const {
    return x >= 0 && y >= 0 && x + y <= (kind == KV ? n : n - 1);
  }
};

template <class P>
__device__ __forceinline__ typename P::W wget(const StencilPtr& st, int64_t i) {
  return P::weight(st, i);
}

// One row: sum_k w_k x[nb_k], over the valid neighbours when `check`.
template <class P, int NN>
__device__ __forceinline__ typename P::T row(const typename P::T* __restrict__ xm, const Geo& G, const NbD* nb,
                                             const StencilPtr& st, int64_t wbase, int x, int y, bool check) {
  typename P::Acc1 a;
  P::first1(a, wget<P>(st, wbase), P::load(xm + G.idx(nb[0].kind, x + nb[0].dx, y + nb[0].dy)));
#pragma unroll
  for (int k = 1; k < NN; ++k) {
    const int kx = x + nb[k].dx, ky = y + nb[k].dy;
    if (check && !G.valid(nb[k].kind, kx, ky)) continue;
    P::add1(a, wget<P>(st, wbase + k), P::load(xm + G.idx(nb[k].kind, kx, ky)));
  }
  return P::finish1(a);
}

template <class P>
__global__ void __launch_bounds__(128) k_p2_apply(const typename P::T* __restrict__ x, typename P::T* __restrict__ y,
                                                  Geo G, StencilPtr st) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y;
  const int n = G.n;
  if (px > n - py) return;
  const int64_t cell = blockIdx.z;
  const typename P::T* __restrict__ xm = x + cell * G.S2;
  typename P::T* __restrict__ ym = y + cell * G.S2;
  const int64_t wb = cell * P2W;
  // vertex row; the first neighbour of every list is valid for every DoF of
  // its kind, so it starts the sum unchecked
  {
    const int cls = (px == 0 ? 1 : 0) | (py == 0 ? 2 : 0) | (px + py == n ? 4 : 0);
    ym[G.vidx(px, py)] = row<P, P2_NV>(xm, G, c_nbv, st, wb + cls * P2_NV, px, py, cls != 0);
  }
  if (px + py <= n - 1) {
    const int bnd[3] = {py == 0, px == 0, px + py == n - 1};
#pragma unroll
    for (int g = 0; g < 3; ++g)
      ym[G.eidx(g, px, py)] = row<P, P2_NE>(xm, G, c_nbe[g], st, wb + P2_EOFF + (g * 2 + bnd[g]) * P2_NE, px, py,
                                            bnd[g] != 0);
  }
}

// Edge DoFs on coarse edges: sum the copies' partial rows in ascending macro
// order and write the sum to every copy (Dirichlet edges: y = x).
template <class T>
__global__ void __launch_bounds__(128) k_p2_edge_reduce(const T* __restrict__ x, T* __restrict__ y,
                                                        const int4* __restrict__ items, const Prim* __restrict__ prims,
                                                        const Inc* __restrict__ incs, Geo G) {
  const int4 it = items[blockIdx.x];
  const int t = it.y + threadIdx.x;
  if (t >= it.z) return;
  const Prim p = prims[it.x];
  if (!p.boundary && p.inc_count == 1) return;
  const int n = G.n;
  // slot of micro-edge t (counted from the canonical low vertex) in copy i
  auto slot_of = [&](int i) -> int64_t {
    const Inc inc = incs[p.inc_begin + i];
    const int a = inc.corner[0], b = inc.corner[1];
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int tl = (a == lo) ? t : n - 1 - t;  // counted from the lower local corner
    int g, ex, ey;
    if (lo == 0 && hi == 1) {
      g = 0, ex = tl, ey = 0;  // X, y = 0, from corner 0
    } else if (lo == 0 && hi == 2) {
      g = 1, ex = 0, ey = tl;  // Y, x = 0, from corner 0
    } else {
      g = 2, ex = n - 1 - tl, ey = tl;  // XY, x + y = n - 1, from corner 1
    }
    return (int64_t)inc.cell * G.S2 + G.eidx(g, ex, ey);
  };
  T acc = T(0);
  if (p.boundary) {
    acc = __ldg(x + slot_of(0));
  } else {
    for (int i = 0; i < p.inc_count; ++i) acc += y[slot_of(i)];
  }
  for (int i = 0; i < p.inc_count; ++i) y[slot_of(i)] = acc;
}

// Vertex DoFs on coarse vertices and edges: as the P1 reduction, in the P2
// macro blocks.
template <class T>
__global__ void __launch_bounds__(128) k_p2_vertex_reduce(const T* __restrict__ x, T* __restrict__ y,
                                                          const int4* __restrict__ items, const Prim* __restrict__ prims,
                                                          const Inc* __restrict__ incs, Geo G) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  if (!p.boundary && p.inc_count == 1) return;
  const int n = G.n;
  int wv[2] = {0, 0};
  if (p.type == 0) {
    wv[0] = n;
  } else {
    wv[0] = n - a;
    wv[1] = a;
  }
  auto slot_of = [&](int i) -> int64_t {
    const Inc inc = incs[p.inc_begin + i];
    int q[2] = {0, 0};
    for (int j = 0; j <= p.type; ++j)
      if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
    return (int64_t)inc.cell * G.S2 + G.vidx(q[0], q[1]);
  };
  T acc = T(0);
  if (p.boundary) {
    acc = __ldg(x + slot_of(0));
  } else {
    for (int i = 0; i < p.inc_count; ++i) acc += y[slot_of(i)];
  }
  for (int i = 0; i < p.inc_count; ++i) y[slot_of(i)] = acc;
}

template <class P>
cudaError_t launch_t(const Mesh& m, const LevelDev& L, const void* x, void* y, cudaStream_t s, cudaEvent_t ev_mid,
                     const char** what) {
  using T = typename P::T;
  Geo G;
  G.n = L.n;
  G.Sv = L.slots_per_macro;
  G.Se = p2_edge_slots(L.level);
  G.S2 = G.Sv + 3 * G.Se;
  StencilPtr st{L.p2_st64, L.p2_st32, L.p2_hi, L.p2_lo};
  *what = "P2 apply kernel";
  const dim3 grid((unsigned)((L.n + 1 + 127) / 128), (unsigned)(L.n + 1), (unsigned)m.n_cells);
  k_p2_apply<P><<<grid, 128, 0, s>>>((const T*)x, (T*)y, G, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev_mid && (e = cudaEventRecord(ev_mid, s)) != cudaSuccess) return e;
  *what = "P2 interface kernels";
  if (L.n_items > 0)
    k_p2_vertex_reduce<T><<<L.n_items, 128, 0, s>>>((const T*)x, (T*)y, L.items, m.d_prims, m.d_incs, G);
  if (L.n_p2_items > 0)
    k_p2_edge_reduce<T><<<L.n_p2_items, 128, 0, s>>>((const T*)x, (T*)y, L.p2_items, m.d_prims, m.d_incs, G);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_p2_apply(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                            cudaEvent_t ev_mid, const char** what) {
  const LevelDev& L = m.levels[level];
  switch (dtype) {
    case 1: return launch_t<ArF64FF>(m, L, x, y, s, ev_mid, what);
    case 2: return launch_t<ArF32>(m, L, x, y, s, ev_mid, what);
    case 3: return launch_t<ArF64Native>(m, L, x, y, s, ev_mid, what);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
