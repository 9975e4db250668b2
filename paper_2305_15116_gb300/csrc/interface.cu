// Interface step of the 3D apply: completes the DoFs on macro vertices,
// edges and faces.
//
// The paper hands the points on the macro boundary to separate "interface
// primitives" (Sec. 5.1).  Here every copy of such a point in an incident
// macro holds its macro's PARTIAL row (the stencil restricted to the
// micro-elements of that macro, written by the 3D kernels); the partials of
// all incident macros are summed in ascending macro order — a fixed order,
// so the result is deterministic — and the sum is written to every copy.  In
// exact arithmetic the sum is the assembled matrix row.  Points on the
// domain boundary get the Dirichlet identity row: y = x.  (2D computes its
// interface points inside the apply launch, interior2d.cu.)
//
// Work list: one block per item (primitive, row b, points a0..a1-1) of at most
// 128 points; a vertex item has one point.
#include <algorithm>

#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

__device__ __forceinline__ int64_t tri_slot(int n, int x, int y) {
  return (int64_t)y * (n + 2) - ((int64_t)y * (y + 1)) / 2 + x;
}
__device__ __forceinline__ int64_t tet_slot(int n, int x, int y, int z) {
  const int64_t N = n + 1, b = N - z;
  const int64_t zs = N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6;
  return zs + (int64_t)y * b - ((int64_t)y * (y - 1)) / 2 + x;
}

// Slots of every copy of every interface point, in work-list order: item i
// owns the entries from item_base[i], (a - a0) * inc_count + copy for its
// point a.  Built once per level; the reduction then reads the slots instead
// of recomputing them from the incidence tables.
template <int DIM>
__global__ void __launch_bounds__(128) k_build_iface_slots(int64_t* __restrict__ out,
                                                           const int64_t* __restrict__ item_base,
                                                           const int64_t* __restrict__ flat_base,
                                                           longlong2* __restrict__ pairs,
                                                           const int4* __restrict__ items,
                                                           const Prim* __restrict__ prims,
                                                           const Inc* __restrict__ incs, int n, int64_t S) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  const int b = it.y;
  int wv[3] = {0, 0, 0};
  if (p.type == 0) {
    wv[0] = n;
  } else if (p.type == 1) {
    wv[0] = n - a;
    wv[1] = a;
  } else {
    wv[0] = n - a - b;
    wv[1] = a;
    wv[2] = b;
  }
  int64_t* o = out + item_base[blockIdx.x] + (int64_t)(a - it.z) * p.inc_count;
  int64_t s01[2] = {-1, -2};
  for (int i = 0; i < p.inc_count; ++i) {
    const Inc inc = incs[p.inc_begin + i];
    int q[3] = {0, 0, 0};
    for (int j = 0; j <= p.type; ++j)
      if (inc.corner[j] >= 1) q[inc.corner[j] - 1] += wv[j];
    o[i] = (int64_t)inc.cell * S + (DIM == 2 ? tri_slot(n, q[0], q[1]) : tet_slot(n, q[0], q[1], q[2]));
    if (i < 2) s01[i] = o[i];
  }
  // points of two copies (inside the domain) or one (Dirichlet) also go to
  // the flat pair table: (slot, slot) or (slot, -2)
  const int64_t fb = flat_base[blockIdx.x];
  if (fb >= 0) pairs[fb + (a - it.z)] = make_longlong2(s01[0], p.boundary ? -2 : s01[1]);
}

// Reduction with the precomputed tables, one launch.  Blocks [0, rest_blocks)
// take the points with three or more copies (edges and vertices), two items of
// the rest list per block: the copies' partial rows are summed in ascending
// macro order (the slot table's order) and the sum written into every copy; a
// Dirichlet point gets y = x.  The other blocks take the pair table, one
// thread per point: two copies are summed (lower macro first) and the sum
// written to both, or a Dirichlet point of one copy gets y = x.  Pair blocks
// run in table order, so that the points in flight at any time lie close
// together in the vectors.  The two sets of points are disjoint.
template <class T>
__global__ void __launch_bounds__(256) k_interface_reduce_flat(const T* __restrict__ x, T* __restrict__ y,
                                                               const longlong2* __restrict__ pairs, int64_t n_pairs,
                                                               const int4* __restrict__ items,
                                                               const Prim* __restrict__ prims,
                                                               const int64_t* __restrict__ item_base,
                                                               const int64_t* __restrict__ slots,
                                                               const int* __restrict__ list, int n_rest,
                                                               int rest_blocks) {
  if ((int)blockIdx.x < rest_blocks) {
    const int k = 2 * (int)blockIdx.x + (int)(threadIdx.x >> 7);
    if (k >= n_rest) return;
    const int item = list[k];
    const int4 it = items[item];
    const int a = it.z + (int)(threadIdx.x & 127);
    if (a >= it.w) return;
    const Prim p = prims[it.x];
    if (!p.boundary && p.inc_count == 1) return;
    const int64_t* sl = slots + item_base[item] + (int64_t)(a - it.z) * p.inc_count;
    T acc = T(0);
    if (p.boundary) {
      acc = __ldg(x + __ldg(sl));
    } else {
      for (int i = 0; i < p.inc_count; ++i) acc += y[__ldg(sl + i)];
    }
    for (int i = 0; i < p.inc_count; ++i) y[__ldg(sl + i)] = acc;
    return;
  }
  const int64_t i = (int64_t)(blockIdx.x - rest_blocks) * blockDim.x + threadIdx.x;
  if (i >= n_pairs) return;
  const longlong2 pr = pairs[i];
  if (pr.y == -2) {
    y[pr.x] = __ldg(x + pr.x);
  } else {
    const T v = y[pr.x] + y[pr.y];
    y[pr.x] = v;
    y[pr.y] = v;
  }
}

// Reduce variant: the copies already hold their macro's partial row (written
// by the 3D slab kernel); sum them in ascending macro order and write the sum
// into every copy.  A point with a single copy is already complete.
template <class T, int DIM>
__global__ void __launch_bounds__(128) k_interface_reduce(const T* __restrict__ x, T* __restrict__ y,
                                                          const int4* __restrict__ items,
                                                          const Prim* __restrict__ prims,
                                                          const Inc* __restrict__ incs, int n, int64_t S) {
  const int4 it = items[blockIdx.x];
  const int a = it.z + threadIdx.x;
  if (a >= it.w) return;
  const Prim p = prims[it.x];
  if (!p.boundary && p.inc_count == 1) return;
  const int b = it.y;
  int wv[3] = {0, 0, 0};
  if (p.type == 0) {
    wv[0] = n;
  } else if (p.type == 1) {
    wv[0] = n - a;
    wv[1] = a;
  } else {
    wv[0] = n - a - b;
    wv[1] = a;
    wv[2] = b;
  }
  const int nverts = p.type + 1;
  // slot of this point in the i-th incident cell
  auto slot_of = [&](int i) -> int64_t {
    const Inc inc = incs[p.inc_begin + i];
    int q[3] = {0, 0, 0};
    for (int j = 0; j < nverts; ++j) {
      const int c = inc.corner[j];
      if (c >= 1) q[c - 1] += wv[j];
    }
    return (int64_t)inc.cell * S + (DIM == 2 ? tri_slot(n, q[0], q[1]) : tet_slot(n, q[0], q[1], q[2]));
  };
  T acc = T(0);
  if (p.boundary) {
    acc = __ldg(x + slot_of(0));
  } else {
    for (int i = 0; i < p.inc_count; ++i) acc += y[slot_of(i)];
  }
  for (int i = 0; i < p.inc_count; ++i) y[slot_of(i)] = acc;
}

template <class T>
cudaError_t launch_reduce_t(int dim, const Mesh& m, const LevelDev& L, const void* x, void* y, cudaStream_t s) {
  if (L.n_items == 0) return cudaSuccess;
  if (L.if_slots) {
    const int rest_blocks = (L.n_if_rest + 1) / 2;
    const int64_t blocks = rest_blocks + (L.n_if_pairs + 255) / 256;
    if (blocks > 0)
      k_interface_reduce_flat<T><<<(unsigned)blocks, 256, 0, s>>>((const T*)x, (T*)y, L.if_pairs, L.n_if_pairs,
                                                                  L.items, m.d_prims, L.if_item_base, L.if_slots,
                                                                  L.if_rest, L.n_if_rest, rest_blocks);
    return cudaGetLastError();
  }
  if (dim == 2)
    k_interface_reduce<T, 2><<<L.n_items, 128, 0, s>>>((const T*)x, (T*)y, L.items, m.d_prims, m.d_incs, L.n,
                                                        L.slots_per_macro);
  else
    k_interface_reduce<T, 3><<<L.n_items, 128, 0, s>>>((const T*)x, (T*)y, L.items, m.d_prims, m.d_incs, L.n,
                                                        L.slots_per_macro);
  return cudaGetLastError();
}

}  // namespace

cudaError_t build_iface_slots(const Mesh& m, const LevelDev& L, cudaStream_t s) {
  if (L.n_items == 0 || !L.if_slots) return cudaSuccess;
  if (m.dim == 2)
    k_build_iface_slots<2><<<L.n_items, 128, 0, s>>>(L.if_slots, L.if_item_base, L.if_flat_base, L.if_pairs,
                                                      L.items, m.d_prims, m.d_incs, L.n, L.slots_per_macro);
  else
    k_build_iface_slots<3><<<L.n_items, 128, 0, s>>>(L.if_slots, L.if_item_base, L.if_flat_base, L.if_pairs,
                                                      L.items, m.d_prims, m.d_incs, L.n, L.slots_per_macro);
  return cudaGetLastError();
}

cudaError_t launch_interface_reduce(int dtype, int dim, const Mesh& m, const LevelDev& L, const void* x, void* y,
                                    cudaStream_t s) {
  switch (dtype) {
    case 1:
    case 3: return launch_reduce_t<double>(dim, m, L, x, y, s);
    case 2: return launch_reduce_t<float>(dim, m, L, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_apply(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                         cudaEvent_t ev_mid, const char** what) {
  const LevelDev& L = m.levels[level];
  if (dtype == 1 && !L.ff_ok) dtype = 3;  // weights outside the float-float range: native fp64
  cudaError_t e;
  if (m.dim == 2) {
    // one launch: macro-interior tiles and interface points side by side
    *what = "2D apply kernel";
    e = launch_apply2d(dtype, m, L, x, y, s);
    if (e != cudaSuccess) return e;
    if (ev_mid) {
      *what = "cudaEventRecord";
      e = cudaEventRecord(ev_mid, s);
    }
    return e;
  }
  // 3D: the slab kernel (n <= 64: whole slices in shared memory) or the row
  // kernel (larger levels) writes every slot, partial rows at macro
  // boundaries included; the interface step then reduces the copies
  *what = "3D kernel";
  e = L.n_slabs > 0 ? launch_slab3d(dtype, L, x, y, s) : launch_row3d(dtype, L, m.n_cells, x, y, s);
  if (e != cudaSuccess) return e;
  if (ev_mid) {
    *what = "cudaEventRecord";
    e = cudaEventRecord(ev_mid, s);
    if (e != cudaSuccess) return e;
  }
  *what = "interface reduce kernel";
  return launch_interface_reduce(dtype, m.dim, m, L, x, y, s);
}

cudaError_t launch_apply_partial(const Mesh& m, int level, int dtype, const void* x, void* y, cudaStream_t s,
                                 const char** what) {
  const LevelDev& L = m.levels[level];
  if (dtype == 1 && !L.ff_ok) dtype = 3;  // weights outside the float-float range: native fp64
  if (m.dim == 2) {
    *what = "2D apply kernel (partial rows)";
    return launch_apply2d_partial(dtype, m, L, x, y, s);
  }
  // 3D: the slab or row kernel writes the partial rows; no reduction
  *what = "3D kernel";
  return L.n_slabs > 0 ? launch_slab3d(dtype, L, x, y, s) : launch_row3d(dtype, L, m.n_cells, x, y, s);
}

}  // namespace hyteg
