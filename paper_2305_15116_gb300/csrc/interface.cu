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
#include <vector>

#include "arith.cuh"
#include "group.cuh"
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
// together in the vectors.  The two sets of points are disjoint.  A body of
// group.cuh: one launch serves one mesh or a group.
template <class T>
struct ReduceFlat {
  static constexpr int kThreads = 256;
  static constexpr bool kLateWait = true;  // the items' tables first
  struct Prm {
    const T* x;
    T* y;
    const longlong2* pairs;
    int64_t n_pairs;
    const int4* items;
    const Prim* prims;
    const int64_t *item_base, *slots;
    const int* list;
    int n_rest, rest_blocks;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int) {
    if (block < p.rest_blocks) {
      const int k = 2 * block + (int)(threadIdx.x >> 7);
      if (k >= p.n_rest) return;
      const int item = p.list[k];
      const int4 it = p.items[item];
      const int t = (int)(threadIdx.x & 127);
      const Prim pr = p.prims[it.x];
      if (!pr.boundary && pr.inc_count == 1) return;
      pdl_wait();
      if (pr.type == 0 && !pr.boundary && pr.inc_count <= 32) {
        // a coarse vertex inside the domain: lane i of the item's first warp
        // takes copy i, and every lane adds the copies in ascending order
        // (the order of the loop below) through shuffles
        if (t >= 32) return;
        const int64_t* sl = p.slots + p.item_base[item];
        const bool mine = t < pr.inc_count;
        const int64_t s = mine ? __ldg(sl + t) : 0;
        const T v = mine ? p.y[s] : T(0);
        T acc = T(0);
        for (int i = 0; i < pr.inc_count; ++i) acc += __shfl_sync(0xFFFFFFFFu, v, i);
        if (mine) p.y[s] = acc;
        return;
      }
      const int a = it.z + t;
      if (a >= it.w) return;
      const int64_t* sl = p.slots + p.item_base[item] + (int64_t)(a - it.z) * pr.inc_count;
      T acc = T(0);
      if (pr.boundary) {
        acc = __ldg(p.x + __ldg(sl));
      } else {
        // the copies' loads four at a time, added in ascending order
        int i = 0;
        for (; i + 4 <= pr.inc_count; i += 4) {
          const int64_t s0 = __ldg(sl + i), s1 = __ldg(sl + i + 1), s2 = __ldg(sl + i + 2), s3 = __ldg(sl + i + 3);
          const T v0 = p.y[s0], v1 = p.y[s1], v2 = p.y[s2], v3 = p.y[s3];
          acc += v0;
          acc += v1;
          acc += v2;
          acc += v3;
        }
        for (; i < pr.inc_count; ++i) acc += p.y[__ldg(sl + i)];
      }
      for (int i = 0; i < pr.inc_count; ++i) p.y[__ldg(sl + i)] = acc;
      return;
    }
    const int64_t i = (int64_t)(block - p.rest_blocks) * 256 + threadIdx.x;
    if (i >= p.n_pairs) return;
    const longlong2 pr = p.pairs[i];
    pdl_wait();
    if (pr.y == -2) {
      p.y[pr.x] = __ldg(p.x + pr.x);
    } else {
      const T v = p.y[pr.x] + p.y[pr.y];
      p.y[pr.x] = v;
      p.y[pr.y] = v;
    }
  }
};

// Reduce variant without the tables (2D levels): the copies already hold
// their macro's partial row; sum them in ascending macro order and write the
// sum into every copy.  A point with a single copy is already complete.
template <class T, int DIM>
struct ReduceItems {
  static constexpr int kThreads = 128;
  static constexpr bool kLateWait = true;  // the items' tables first
  struct Prm {
    const T* x;
    T* y;
    const int4* items;
    const Prim* prims;
    const Inc* incs;
    int n;
    int64_t S;
  };
  static __device__ __forceinline__ void run(const Prm& p, int block, int) {
    const int4 it = p.items[block];
    const Prim pr = p.prims[it.x];
    if (!pr.boundary && pr.inc_count == 1) return;
    const int n = p.n;
    pdl_wait();
    if (pr.type == 0 && !pr.boundary && pr.inc_count <= 32) {
      // a coarse vertex inside the domain: lane i of the first warp takes
      // copy i, added in ascending copy order through shuffles
      if (threadIdx.x >= 32) return;
      const bool mine = (int)threadIdx.x < pr.inc_count;
      int64_t s = 0;
      if (mine) {
        const Inc inc = p.incs[pr.inc_begin + threadIdx.x];
        int q[3] = {0, 0, 0};
        if (inc.corner[0] >= 1) q[inc.corner[0] - 1] += n;
        s = (int64_t)inc.cell * p.S + (DIM == 2 ? tri_slot(n, q[0], q[1]) : tet_slot(n, q[0], q[1], q[2]));
      }
      const T v = mine ? p.y[s] : T(0);
      T acc = T(0);
      for (int i = 0; i < pr.inc_count; ++i) acc += __shfl_sync(0xFFFFFFFFu, v, i);
      if (mine) p.y[s] = acc;
      return;
    }
    const int a = it.z + threadIdx.x;
    if (a >= it.w) return;
    const int b = it.y;
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
    const int nverts = pr.type + 1;
    // slot of this point in the i-th incident cell
    auto slot_of = [&](int i) -> int64_t {
      const Inc inc = p.incs[pr.inc_begin + i];
      int q[3] = {0, 0, 0};
      for (int j = 0; j < nverts; ++j) {
        const int c = inc.corner[j];
        if (c >= 1) q[c - 1] += wv[j];
      }
      return (int64_t)inc.cell * p.S + (DIM == 2 ? tri_slot(n, q[0], q[1]) : tet_slot(n, q[0], q[1], q[2]));
    };
    T acc = T(0);
    if (pr.boundary) {
      acc = __ldg(p.x + slot_of(0));
    } else {
      for (int i = 0; i < pr.inc_count; ++i) acc += p.y[slot_of(i)];
    }
    for (int i = 0; i < pr.inc_count; ++i) p.y[slot_of(i)] = acc;
  }
};

template <class T, int DIM>
cudaError_t reduce_items(const Mesh* const* ms, const int* levels, const void* const* x, void* const* y, int cnt,
                         cudaStream_t s) {
  std::vector<typename ReduceItems<T, DIM>::Prm> p;
  std::vector<int> blocks;
  for (int i = 0; i < cnt; ++i) {
    const LevelDev& L = ms[i]->levels[levels[i]];
    p.push_back({(const T*)x[i], (T*)y[i], L.items, ms[i]->d_prims, ms[i]->d_incs, L.n, L.slots_per_macro});
    blocks.push_back(L.n_items);
  }
  return launch_group<ReduceItems<T, DIM>>(p.data(), blocks.data(), cnt, s);
}

// The interface reduction of every mesh of a group (the same dimension), one
// launch per kind of table: the flat tables where the level has them (3D),
// else the item list.
template <class T>
cudaError_t launch_reduce_group_t(const Mesh* const* ms, const int* levels, const void* const* x, void* const* y,
                                  int cnt, cudaStream_t s) {
  std::vector<typename ReduceFlat<T>::Prm> pf;
  std::vector<int> bf;
  std::vector<const Mesh*> mi;
  std::vector<int> li;
  std::vector<const void*> xi;
  std::vector<void*> yi;
  for (int i = 0; i < cnt; ++i) {
    const Mesh& m = *ms[i];
    const LevelDev& L = m.levels[levels[i]];
    if (L.n_items == 0) continue;
    if (L.if_slots) {
      const int rest_blocks = (L.n_if_rest + 1) / 2;
      const int64_t blocks = rest_blocks + (L.n_if_pairs + 255) / 256;
      if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
      pf.push_back({(const T*)x[i], (T*)y[i], L.if_pairs, L.n_if_pairs, L.items, m.d_prims, L.if_item_base,
                    L.if_slots, L.if_rest, L.n_if_rest, rest_blocks});
      bf.push_back(int(blocks));
    } else {
      mi.push_back(ms[i]);
      li.push_back(levels[i]);
      xi.push_back(x[i]);
      yi.push_back(y[i]);
    }
  }
  if (!pf.empty()) {
    const cudaError_t e = launch_group<ReduceFlat<T>>(pf.data(), bf.data(), int(pf.size()), s);
    if (e != cudaSuccess) return e;
  }
  if (mi.empty()) return cudaSuccess;
  const int k = int(mi.size());
  return ms[0]->dim == 2 ? reduce_items<T, 2>(mi.data(), li.data(), xi.data(), yi.data(), k, s)
                         : reduce_items<T, 3>(mi.data(), li.data(), xi.data(), yi.data(), k, s);
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

cudaError_t launch_interface_reduce_group(int dtype, const Mesh* const* ms, const int* levels, const void* const* x,
                                          void* const* y, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  switch (dtype) {
    case 1:
    case 3: return launch_reduce_group_t<double>(ms, levels, x, y, count, s);
    case 2: return launch_reduce_group_t<float>(ms, levels, x, y, count, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_interface_reduce(int dtype, const Mesh& m, int level, const void* x, void* y, cudaStream_t s) {
  const Mesh* mp = &m;
  return launch_interface_reduce_group(dtype, &mp, &level, &x, &y, 1, s);
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
  return launch_interface_reduce(dtype, m, level, x, y, s);
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
