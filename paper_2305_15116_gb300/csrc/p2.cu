// P2 operator apply (2D): the vertex-to-vertex, edge-to-vertex,
// vertex-to-edge and edge-to-edge kernels of Sec. 5.2-5.5 merged into one
// pass, as the paper proposes for its next step (Sec. 7: one kernel instead
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
#include <type_traits>

#include "arith.cuh"
#include "fallback.cuh"
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
// A float-float row that read an input outside the float-float range
// (arith.cuh) is recomputed in native fp64 from memory.
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
  if constexpr (P::kPoison) {
    if (P::bad1(a)) return row<ArF64Native, NN>(xm, G, nb, st, wbase, x, y, true);
  }
  return P::finish1(a);
}

// DoFs on the macro's edges: every lattice point on the macro boundary or
// next to its long edge, one thread each, evaluates those of its DoFs whose
// class is not interior, with the class's partial stencil; neighbours outside
// the macro carry weight 0 and are not read.  Points of one macro: row y = 0
// (x = 0..n), column x = 0 (y = 1..n), the long edge x + y = n (x = 1..n-1)
// and the line x + y = n-1 (x = 1..n-2).
template <class P>
__global__ void __launch_bounds__(128) k_p2_boundary(const typename P::T* __restrict__ x,
                                                     typename P::T* __restrict__ y, Geo G, StencilPtr st,
                                                     int n_points) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_points) return;
  const int n = G.n;
  int px, py;
  if (i <= n) {
    px = i, py = 0;
  } else if (i <= 2 * n) {
    px = 0, py = i - n;
  } else if (i < 3 * n) {
    px = i - 2 * n, py = n - px;
  } else {
    px = i - 3 * n + 1, py = n - 1 - px;
  }
  const int64_t cell = blockIdx.y;
  const typename P::T* __restrict__ xm = x + cell * G.S2;
  typename P::T* __restrict__ ym = y + cell * G.S2;
  const int64_t wb = cell * P2W;
  const int cls = (px == 0 ? 1 : 0) | (py == 0 ? 2 : 0) | (px + py == n ? 4 : 0);
  // the first neighbour of every list is valid for every DoF of its kind
  if (cls != 0) ym[G.vidx(px, py)] = row<P, P2_NV>(xm, G, c_nbv, st, wb + cls * P2_NV, px, py, true);
  if (px + py <= n - 1) {
    const bool bnd[3] = {py == 0, px == 0, px + py == n - 1};
#pragma unroll
    for (int g = 0; g < 3; ++g)
      if (bnd[g])
        ym[G.eidx(g, px, py)] = row<P, P2_NE>(xm, G, c_nbe[g], st, wb + P2_EOFF + (g * 2 + 1) * P2_NE, px, py, true);
  }
}

// ---- row kernel for the macro-interior DoFs -----------------------------------
// One warp per tile of 32 lattice columns (30 written) and up to 64 rows of one
// macro, walking up the rows as the P1 kernel does: every lane stages its
// column of the next rows of all four arrays with cp.async, keeps three rows
// of each array in registers (with the x-1 / x+1 neighbours fetched once per
// row by warp shuffles) and evaluates the four DoFs of its lattice point
// whose class is interior:
//   V(x,y): x >= 1, y >= 1, x + y <= n-1     X(x,y): y >= 1, x + y <= n-1
//   Y(x,y): x >= 1, x + y <= n-1              XY(x,y): x + y <= n-2
// The DoFs on the macro's edges (their partial rows) come from k_p2_boundary.
// For the Laplacian the coupling of a vertex with the edge opposite to it in
// a triangle vanishes: integral of (4 lambda_i - 1) lambda_k is
// 4|T|/12 - |T|/3 = 0.  The host sets those weights to zero (6 of the 12 edge
// terms of a vertex row, 2 of the 4 vertex terms of an edge row) and this
// kernel skips them: 34 products per lattice point instead of 46.

// One row r of the four arrays seen from one lane (column c): own values,
// their right (x+1, "e") and left (x-1, "w") neighbours where a stencil needs them.
template <class P>
struct P2Row {
  typename P::V vc, ve, vw, xc, xw, yc, ye, yw, dc, dw;
};

template <class P>
__device__ __forceinline__ P2Row<P> make_p2row(typename P::V v, typename P::V ex, typename P::V ey,
                                               typename P::V ed) {
  P2Row<P> r;
  r.vc = v;
  r.ve = P::down(v);
  r.vw = P::up(v);
  r.xc = ex;
  r.xw = P::up(ex);
  r.yc = ey;
  r.ye = P::down(ey);
  r.yw = P::up(ey);
  r.dc = ed;
  r.dw = P::up(ed);
  return r;
}

// The 46 interior weights of a macro (19 vertex row, 9 per edge group), kept
// in registers for fp32 and in shared memory (one slice per warp) otherwise.
template <class P, bool REG>
struct P2W46;
template <class P>
struct P2W46<P, true> {
  typename P::W w[46];
  __device__ __forceinline__ void init(const StencilPtr& st, int64_t base, typename P::W*) {
#pragma unroll
    for (int k = 0; k < 46; ++k) w[k] = P::weight(st, k < P2_NV ? base + k : base + P2_EOFF + ((k - P2_NV) / P2_NE) * 2 * P2_NE + (k - P2_NV) % P2_NE);
  }
  __device__ __forceinline__ const typename P::W& operator[](int k) const { return w[k]; }
};
template <class P>
struct P2W46<P, false> {
  typename P::W* w;
  __device__ __forceinline__ void init(const StencilPtr& st, int64_t base, typename P::W* slice) {
    w = slice;
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < 46; k += 32)
      w[k] = P::weight(st, k < P2_NV ? base + k : base + P2_EOFF + ((k - P2_NV) / P2_NE) * 2 * P2_NE + (k - P2_NV) % P2_NE);
    __syncwarp();
  }
  __device__ __forceinline__ const typename P::W& operator[](int k) const { return w[k]; }
};

__device__ __forceinline__ void p2_cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
// a shared-memory element of `bytes` (4 or 8) set to zero by an asynchronous
// copy that reads no bytes (src, a valid global address, is not accessed)
__device__ __forceinline__ void p2_cp_zero(void* smem, const void* src, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, 0;" ::"r"(sa), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, 0;" ::"r"(sa), "l"(src));
}
__device__ __forceinline__ void p2_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void p2_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// rows in flight per warp: three, one per register row, so that the walk
// unrolled by three finds every ring slot at a constant (8 rows for fp32 and
// 4 for 8-byte data with a computed slot ran 6 % / 1 % slower)
template <class T>
struct P2Ring {
  static constexpr int value = 3;
};
constexpr int P2THREADS = 256;

template <class P>
__global__ void __launch_bounds__(P2THREADS) k_p2_rows(const typename P::T* __restrict__ x, typename P::T* __restrict__ y,
                                                       const int4* __restrict__ tiles, int n_tiles, int64_t n_warps,
                                                       Geo G, StencilPtr st) {
  using T = typename P::T;
  using V = typename P::V;
  constexpr bool REG = false;  // weights from shared memory: fewer registers, more resident warps
  constexpr int P2RING = P2Ring<T>::value;
  __shared__ T ring_all[P2THREADS / 32][P2RING][4][32];
  __shared__ typename P::W wslice_all[P2THREADS / 32][REG ? 1 : 46];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  T(*ring)[4][32] = ring_all[wid];
  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];
  const int n = G.n;
  const int c = t.x - 1 + lane;  // this lane's lattice column
  const T* __restrict__ xm = x + m * G.S2;
  T* __restrict__ ym = y + m * G.S2;
  P2W46<P, REG> W;
  W.init(st, m * (int64_t)P2W, wslice_all[wid]);

  const int steps = t.z - t.y + 2;  // rows t.y-1 .. t.z
  // row cursors (32-bit offsets inside the macro block): vertex row r at
  // r(n+2) - r(r+1)/2 with n+1-r entries, edge row r at r n - r(r-1)/2 with
  // n-r entries; row -1 is empty and its successor starts at 0
  struct Cur {
    int ov, lv, oe, le;
    __device__ __forceinline__ void init(int n, int r) {
      ov = r * (n + 2) - (r * (r + 1)) / 2;
      lv = n + 1 - r;
      oe = r * n - (r * (r - 1)) / 2;
      le = n - r;
    }
    __device__ __forceinline__ void next() {
      ov += lv;
      lv -= 1;
      oe += le;
      le -= 1;
    }
  };
  const int se = (int)G.Se, sv = (int)G.Sv;
  Cur cs;  // next row to stage
  cs.init(n, t.y - 1);
  int rs = t.y - 1;
  auto stage = [&](int slot) {
    if (rs >= 0) {
      if (c >= 0 && c < cs.lv) p2_cp_async(&ring[slot][0][lane], xm + cs.ov + c, sizeof(T));
      if (c >= 0 && c < cs.le) {
        const T* e0 = xm + sv + cs.oe + c;
        p2_cp_async(&ring[slot][1][lane], e0, sizeof(T));
        p2_cp_async(&ring[slot][2][lane], e0 + se, sizeof(T));
        p2_cp_async(&ring[slot][3][lane], e0 + 2 * se, sizeof(T));
      }
    }
    ++rs;
    cs.next();
  };
  if constexpr (P::kPoison) {
    // Float-float: the ring starts zeroed (copies that read nothing, completed
    // before the first row is staged) and a value outside a row is not
    // selected away: it is zero or an input of an earlier row, met only by
    // zero weights, and one outside the float-float range marks the row,
    // which is then recomputed in native fp64.
#pragma unroll
    for (int k = 0; k < P2RING; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) p2_cp_zero(&ring[k][j][lane], xm, sizeof(T));
    p2_commit();
    p2_wait<0>();
  }
#pragma unroll
  for (int k = 0; k < P2RING; ++k) {
    if (k < steps) stage(k);
    p2_commit();
  }
  Cur cr;  // row being consumed
  cr.init(n, t.y - 1);
  int rc = t.y - 1;
  auto take = [&](int k, auto slot_c) -> P2Row<P> {
    p2_wait<P2RING - 1>();
    constexpr int slot = decltype(slot_c)::value;
    const bool okv = P::kPoison || (rc >= 0 && c >= 0 && c < cr.lv),
               oke = P::kPoison || (rc >= 0 && c >= 0 && c < cr.le);
    const V v = okv ? P::conv(ring[slot][0][lane]) : P::zero();
    const V ex = oke ? P::conv(ring[slot][1][lane]) : P::zero();
    const V ey = oke ? P::conv(ring[slot][2][lane]) : P::zero();
    const V ed = oke ? P::conv(ring[slot][3][lane]) : P::zero();
    if (k + P2RING < steps) stage(slot);
    p2_commit();
    ++rc;
    cr.next();
    return make_p2row<P>(v, ex, ey, ed);
  };
  const bool writer = lane >= 1 && lane <= 30;
  int yo = t.y;  // output row
  Cur co;
  co.init(n, t.y);
  typename P::Mark1 mk = P::mark1_0();  // float-float: notes rows that read an input outside the range
  auto step = [&](const P2Row<P>& lo, const P2Row<P>& ce, const P2Row<P>& hi) {
    const int cx = c;
    // vertex row (NBV order)
    if (writer && cx >= 1 && yo >= 1 && cx + yo <= n - 1) {
      typename P::Acc1 a;
      P::first1(a, W[0], ce.vc);
      P::add1(a, W[1], ce.ve);
      P::add1(a, W[2], ce.vw);
      P::add1(a, W[3], hi.vc);
      P::add1(a, W[4], lo.vc);
      P::add1(a, W[5], lo.ve);
      P::add1(a, W[6], hi.vw);
      P::add1(a, W[7], ce.xc);
      P::add1(a, W[8], ce.xw);
      P::add1(a, W[11], ce.yc);
      P::add1(a, W[12], lo.yc);
      P::add1(a, W[16], ce.dw);
      P::add1(a, W[17], lo.dc);
      P::mark1(mk, a);
      ym[co.ov + cx] = P::finish1(a);
    }
    if (writer && cx + yo <= n - 1) {
      T* e0 = ym + sv + co.oe + cx;
      if (yo >= 1) {  // X (NBX order)
        typename P::Acc1 a;
        P::first1(a, W[19], ce.vc);
        P::add1(a, W[20], ce.ve);
        P::add1(a, W[23], ce.xc);
        P::add1(a, W[24], ce.yc);
        P::add1(a, W[25], lo.ye);
        P::add1(a, W[26], ce.dc);
        P::add1(a, W[27], lo.dc);
        P::mark1(mk, a);
        e0[0] = P::finish1(a);
      }
      if (cx >= 1) {  // Y (NBY order)
        typename P::Acc1 a;
        P::first1(a, W[28], ce.vc);
        P::add1(a, W[29], hi.vc);
        P::add1(a, W[32], ce.yc);
        P::add1(a, W[33], ce.xc);
        P::add1(a, W[34], hi.xw);
        P::add1(a, W[35], ce.dc);
        P::add1(a, W[36], ce.dw);
        P::mark1(mk, a);
        e0[se] = P::finish1(a);
      }
      if (cx + yo <= n - 2) {  // XY (NBD order)
        typename P::Acc1 a;
        P::first1(a, W[37], ce.ve);
        P::add1(a, W[38], hi.vc);
        P::add1(a, W[41], ce.dc);
        P::add1(a, W[42], ce.xc);
        P::add1(a, W[43], hi.xc);
        P::add1(a, W[44], ce.yc);
        P::add1(a, W[45], ce.ye);
        P::mark1(mk, a);
        e0[2 * se] = P::finish1(a);
      }
    }
    ++yo;
    co.next();
  };
  using S0 = std::integral_constant<int, 0>;
  using S1 = std::integral_constant<int, 1>;
  using S2 = std::integral_constant<int, 2>;
  P2Row<P> r0 = take(0, S0{});
  P2Row<P> r1 = take(1, S1{});
  P2Row<P> r2;
  for (int k = 2; k < steps; k += 3) {
    r2 = take(k, S2{});
    step(r0, r1, r2);
    if (k + 1 >= steps) break;
    r0 = take(k + 1, S0{});
    step(r1, r2, r0);
    if (k + 2 >= steps) break;
    r1 = take(k + 2, S1{});
    step(r2, r0, r1);
  }
  p2_wait<0>();
  if constexpr (P::kPoison) {
    // rows that read an input outside the float-float range: this lane's
    // column of the tile again, every row it wrote, in native fp64
    if (P::marked1(mk)) {
      const int64_t wv = m * (int64_t)P2W, we = wv + P2_EOFF;
      for (int yy = t.y; yy < t.z; ++yy) {
        if (c >= 1 && yy >= 1 && c + yy <= n - 1)
          ym[G.vidx(c, yy)] = row<ArF64Native, P2_NV>(xm, G, c_nbv, st, wv, c, yy, true);
        if (c + yy <= n - 1) {
          if (yy >= 1) ym[G.eidx(0, c, yy)] = row<ArF64Native, P2_NE>(xm, G, c_nbe[0], st, we, c, yy, true);
          if (c >= 1) ym[G.eidx(1, c, yy)] = row<ArF64Native, P2_NE>(xm, G, c_nbe[1], st, we + 2 * P2_NE, c, yy, true);
          if (c + yy <= n - 2)
            ym[G.eidx(2, c, yy)] = row<ArF64Native, P2_NE>(xm, G, c_nbe[2], st, we + 4 * P2_NE, c, yy, true);
        }
      }
    }
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
  *what = "P2 row kernel";
  cudaError_t e = cudaSuccess;
  if (L.n_p2_tiles > 0) {
    const int64_t n_warps = (int64_t)L.n_p2_tiles * m.n_cells;
    const int64_t blocks = (n_warps * 32 + P2THREADS - 1) / P2THREADS;
    k_p2_rows<P><<<(unsigned)blocks, P2THREADS, 0, s>>>((const T*)x, (T*)y, L.p2_tiles, L.n_p2_tiles, n_warps, G, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  *what = "P2 boundary kernel";
  const int nb = L.n == 1 ? 3 : 4 * L.n - 2;
  k_p2_boundary<P><<<dim3((unsigned)((nb + 127) / 128), (unsigned)m.n_cells), 128, 0, s>>>((const T*)x, (T*)y, G, st,
                                                                                             nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
  if (dtype == 1 && !L.p2_ff_ok) dtype = 3;  // weights outside the float-float range: native fp64
  switch (dtype) {
    case 1: return launch_t<ArF64FF>(m, L, x, y, s, ev_mid, what);
    case 2: return launch_t<ArF32>(m, L, x, y, s, ev_mid, what);
    case 3: return launch_t<ArF64Native>(m, L, x, y, s, ev_mid, what);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
