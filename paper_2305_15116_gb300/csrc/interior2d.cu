// Macro-interior stencil sweep, 2D (the vertex-to-vertex kernel of Sec. 5.2).
//
// For every macro-triangle m and every point strictly inside it
// (x >= 1, y >= 1, x + y <= n - 1):
//   y[x,y] = C x[x,y] + E x[x+1,y] + W x[x-1,y] + N x[x,y+1] + S x[x,y-1]
//          + SE x[x+1,y-1] + NW x[x-1,y+1]
// with the constant weights of macro m.  The triangular array of a macro is
// row-major with x contiguous; row r starts at r(n+2) - r(r+1)/2 and holds
// n+1-r points (Sec. 4).
//
// GPU mapping: one warp per tile of 64 consecutive columns and up to 64 rows;
// the same launch also completes the points on macro vertices and edges (the
// interface step, stencil mode), in blocks of their own.
// Each lane owns two adjacent columns, so it evaluates two points per row and
// the float-float arithmetic of the pair runs on packed f32x2 instructions.
// Each lane stages its two columns of the next RING rows in shared memory with
// cp.async, which keeps RING rows per warp in flight without spending
// registers on them, and keeps three rows in registers (the layer condition
// of Sec. 1.3 held in the register file).  The neighbour columns beyond its
// pair come from the adjacent lanes by warp shuffles, so every value is read
// from memory once per tile plus two halo rows.  62 of the 64 columns are
// written; the outermost two only supply the horizontal halo.
#include <cstdint>
#include <type_traits>
#include <vector>

#include "arith.cuh"
#include "fallback.cuh"
#include "group.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

// One row as seen by a lane that owns the two adjacent columns A = c and
// B = c + 1, packed per term (first half: column A, second half: column B):
// the lane's own values, their right neighbours (B, and A of the next lane)
// and their left neighbours (B of the previous lane, and A).
template <class P>
struct Row {
  typename P::P2 v, e, w;
  typename P::T b[2];  // b at the lane's two points (sweep modes)
};

template <class P>
__device__ __forceinline__ Row<P> make_row(typename P::V a, typename P::V b) {
  const typename P::V right_of_b = P::down(a);  // column c + 2: A of the next lane
  const typename P::V left_of_a = P::up(b);     // column c - 1: B of the previous lane
  Row<P> r;
  r.v = P::pair(a, b);
  r.e = P::pair(b, right_of_b);
  r.w = P::pair(left_of_a, a);
  return r;
}

// Row-walking cursor: offset of row r inside the macro array and its length.
struct Cursor {
  int off;  // r(n+2) - r(r+1)/2
  int len;  // n + 1 - r
  __device__ __forceinline__ void init(int n, int row) {
    off = row * (n + 2) - (row * (row + 1)) / 2;
    len = n + 1 - row;
  }
  __device__ __forceinline__ void next() {
    off += len;
    len -= 1;
  }
};

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
// an 8-byte element of shared memory set to zero by an asynchronous copy that
// reads no bytes (src, a valid global address, is not accessed)
__device__ __forceinline__ void cp_async_zero(void* smem, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, 0;" ::"r"(sa), "l"(src));
}
// a lane's two fp32 columns as one 8-byte-aligned pair
__device__ __forceinline__ bool pair_aligned(const float* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// What a launch writes at a point with (A u) = au:
//   MODE_APPLY:    y = A u
//   MODE_JACOBI:   y = u + omega dinv (b - A u)   (one weighted Jacobi sweep)
//   MODE_RESIDUAL: y = b - A u
// (u = x at the point; b and dinv in the slot layout, copies equal).
//   MODE_PARTIAL:  y = A u inside the macros; at interface points every copy
//                  receives its own macro's partial row instead of the sum
constexpr int MODE_APPLY = 0, MODE_JACOBI = 1, MODE_RESIDUAL = 2, MODE_PARTIAL = 3;

struct ModeArgs {
  const void* b;
  const void* dinv;
  double omega;
};

// sweep modes inside the macro: u, b and dinv of the point come from the
// staged rows
template <int MODE, class T>
__device__ __forceinline__ T mode_out_staged(T au, T u, T b, T d, double omega) {
  if (MODE == MODE_APPLY) return au;
  if (MODE == MODE_RESIDUAL) return b - au;
  return u + (T)omega * d * (b - au);
}

template <int MODE, class T>
__device__ __forceinline__ T mode_out(T au, const T* __restrict__ x, const ModeArgs& md, int64_t i) {
  if (MODE == MODE_APPLY) return au;
  const T bi = __ldg(static_cast<const T*>(md.b) + i);
  if (MODE == MODE_RESIDUAL) return bi - au;
  const T ui = __ldg(x + i), di = __ldg(static_cast<const T*>(md.dinv) + i);
  return ui + (T)md.omega * di * (bi - au);
}

// ---- interface points (coarse vertices and edges), stencil mode ------------
// Each macro holding a copy contributes its partial row (the class stencil of
// the point in that macro: only the macro's own micro-triangles); the partials
// are summed in ascending macro order and the sum is written to every copy.
// Dirichlet points get y = x.  Arithmetic in the element type (fp64 for the
// float-float apply).
__constant__ int c_if_off[NW2][2] = {{0, -1}, {1, -1}, {-1, 0}, {0, 0}, {1, 0}, {-1, 1}, {0, 1}};

__device__ __forceinline__ int64_t if_slot(int n, int x, int y) {
  return (int64_t)y * (n + 2) - ((int64_t)y * (y + 1)) / 2 + x;
}
__device__ __forceinline__ double if_w(const StencilPtr& st, int64_t i, double) { return __ldg(st.d + i); }
__device__ __forceinline__ float if_w(const StencilPtr& st, int64_t i, float) { return __ldg(st.f + i); }
__device__ __forceinline__ double if_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float if_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The partial row of one copy of an interface point: the class stencil of
// the point (local coordinates q) in the copy's macro.
template <class T>
__device__ __forceinline__ T if_partial(const T* __restrict__ x, const Inc& inc, const int q[2], int n, int64_t S,
                                        const StencilPtr& st) {
  const int cls = (q[0] == 0 ? 1 : 0) | (q[1] == 0 ? 2 : 0) | (q[0] + q[1] == n ? 4 : 0);
  const int64_t base = (int64_t)inc.cell * S;
  const int64_t wb = ((int64_t)inc.cell * NCLS2 + cls) * NW2;
  T part = T(0);
#pragma unroll
  for (int k = 0; k < NW2; ++k) {
    const int dx = c_if_off[k][0], dy = c_if_off[k][1];
    if (((cls & 1) && dx < 0) || ((cls & 2) && dy < 0) || ((cls & 4) && dx + dy > 0)) continue;
    part = if_fma(if_w(st, wb + k, T(0)), __ldg(x + base + if_slot(n, q[0] + dx, q[1] + dy)), part);
  }
  return part;
}

template <int MODE, class T>
__device__ __forceinline__ void iface2d_point(const T* __restrict__ x, T* __restrict__ y, const Prim& p, int a,
                                              const Inc* __restrict__ incs, int n, int64_t S, const StencilPtr& st,
                                              const ModeArgs& md) {
  const int wv0 = p.type == 0 ? n : n - a, wv1 = p.type == 0 ? 0 : a;  // weights on the canonical vertices
  auto local = [&](const Inc& inc, int q[2]) {
    q[0] = q[1] = 0;
    if (inc.corner[0] >= 1) q[inc.corner[0] - 1] += wv0;
    if (p.type == 1 && inc.corner[1] >= 1) q[inc.corner[1] - 1] += wv1;
  };
  T acc = T(0);
  if (MODE == MODE_PARTIAL) {  // each copy keeps its own macro's partial row
    for (int i = 0; i < p.inc_count; ++i) {
      const Inc inc = incs[p.inc_begin + i];
      int q[2];
      local(inc, q);
      y[(int64_t)inc.cell * S + if_slot(n, q[0], q[1])] = if_partial(x, inc, q, n, S, st);
    }
    return;
  }
  if (p.boundary) {
    int q[2];
    local(incs[p.inc_begin], q);
    acc = __ldg(x + (int64_t)incs[p.inc_begin].cell * S + if_slot(n, q[0], q[1]));
  } else {
    for (int i = 0; i < p.inc_count; ++i) {
      const Inc inc = incs[p.inc_begin + i];
      int q[2];
      local(inc, q);
      acc += if_partial(x, inc, q, n, S, st);
    }
  }
  if (MODE == MODE_JACOBI || MODE == MODE_RESIDUAL) {  // copies hold equal u, b and dinv: use the first
    int q[2];
    local(incs[p.inc_begin], q);
    acc = mode_out<MODE>(acc, x, md, (int64_t)incs[p.inc_begin].cell * S + if_slot(n, q[0], q[1]));
  }
  for (int i = 0; i < p.inc_count; ++i) {
    const Inc inc = incs[p.inc_begin + i];
    int q[2];
    local(inc, q);
    y[(int64_t)inc.cell * S + if_slot(n, q[0], q[1])] = acc;
  }
}

// A coarse vertex inside the domain (at most 32 incident macros): its copies'
// partial rows are independent, so lane i of one warp takes copy i — walked
// one after another by one thread, the copies' dependent loads were the
// latency floor of the launch on small levels — and every lane adds the
// partials in ascending copy order through shuffles, the order of the serial
// loop, so the result is the same.
template <int MODE, class T>
__device__ __forceinline__ void iface2d_vertex(const T* __restrict__ x, T* __restrict__ y, const Prim& p, int lane,
                                               const Inc* __restrict__ incs, int n, int64_t S, const StencilPtr& st,
                                               const ModeArgs& md) {
  const bool mine = lane < p.inc_count;
  int q[2] = {0, 0};
  int64_t slot = 0;
  T part = T(0);
  if (mine) {
    const Inc inc = incs[p.inc_begin + lane];
    if (inc.corner[0] >= 1) q[inc.corner[0] - 1] += n;
    slot = (int64_t)inc.cell * S + if_slot(n, q[0], q[1]);
    part = if_partial(x, inc, q, n, S, st);
  }
  if (MODE == MODE_PARTIAL) {
    if (mine) y[slot] = part;
    return;
  }
  T acc = T(0);
  for (int i = 0; i < p.inc_count; ++i) acc += __shfl_sync(0xFFFFFFFFu, part, i);
  if (MODE == MODE_JACOBI || MODE == MODE_RESIDUAL)  // copies hold equal u, b and dinv: use the first
    acc = mode_out<MODE>(acc, x, md, __shfl_sync(0xFFFFFFFFu, slot, 0));
  if (mine) y[slot] = acc;
}

// Rows in flight per warp: each lane stages its two columns of the next RING
// rows in shared memory with cp.async, so a warp keeps RING rows outstanding
// without holding them in registers.
constexpr int RING = 3;  // rows in flight; the walk is unrolled by three
constexpr int THREADS2D = 256;

// One launch does the whole apply: blocks 0 .. n_if_blocks-1 take the
// interface items (two items of up to 128 points per block), the others the
// macro-interior tiles.  The two parts write disjoint slots and read only x,
// so they run side by side.
// Threads per block (the sweep modes stage rows of b beside x; the inverse
// diagonal of a macro-interior point is the macro's constant 1 / centre
// weight, so it is not read).
template <int MODE>
struct Thr2 {
  static constexpr int value = THREADS2D;
};

// The work of one block of an apply / sweep launch over one mesh (block =
// the block's index within that mesh's part of the launch).
template <class P, int MODE>
__device__ __forceinline__ void apply2d_block(int block, const typename P::T* __restrict__ x,
                                              typename P::T* __restrict__ y, const int4* __restrict__ tiles,
                                              int n_tiles, int64_t n_warps, int64_t S, int n, const StencilPtr& st,
                                              const int4* __restrict__ items, int n_items,
                                              const Prim* __restrict__ prims, const Inc* __restrict__ incs,
                                              int n_if_blocks, const ModeArgs& md,
                                              typename P::T (*ring_all)[RING][32][2],
                                              typename P::T (*ringb_all)[RING][32][2]) {
  using T = typename P::T;
  constexpr int THR = Thr2<MODE>::value;
  constexpr bool SWEEP = MODE == MODE_JACOBI || MODE == MODE_RESIDUAL;
  static_assert(!SWEEP || sizeof(T) == 4, "the sweep modes are built for fp32");
  if (block < n_if_blocks) {
    const int item = (THR / 128) * block + (int)(threadIdx.x >> 7);
    if (item >= n_items) return;
    const int4 it = items[item];
    const int t = (int)(threadIdx.x & 127);
    const Prim p = prims[it.x];
    pdl_wait();  // the vectors after the previous kernel in the stream (group.cuh)
    if (p.type == 0 && !p.boundary && p.inc_count <= 32) {
      if (t < 32) iface2d_vertex<MODE, T>(x, y, p, t, incs, n, S, st, md);  // the item's first warp
      return;
    }
    const int a = it.z + t;
    if (a < it.w) iface2d_point<MODE, T>(x, y, p, a, incs, n, S, st, md);
    return;
  }
  const int64_t warp = ((int64_t)(block - n_if_blocks) * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  T(*ring)[32][2] = ring_all[threadIdx.x >> 5];
  T(*ringb)[32][2] = ringb_all[SWEEP ? threadIdx.x >> 5 : 0];

  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];
  const int ca = t.x - 1 + 2 * lane;  // column A; column B = ca + 1
  const int cb = ca + 1;
  const T* __restrict__ xm = x + m * S;
  T* __restrict__ ym = y + m * S;
  const T* __restrict__ bm = SWEEP ? static_cast<const T*>(md.b) + m * S : nullptr;
  // inverse diagonal of the macro's interior points, rounded as the set-up's
  const T dint = MODE == MODE_JACOBI ? (T)(1.0 / __ldg(st.d + m * (int64_t)(NCLS2 * NW2) + C2)) : T(0);

  const int64_t wb = m * (int64_t)(NCLS2 * NW2);  // class 0: the full interior stencil
  const typename P::W wSE = P::weight(st, wb + 1), wC = P::weight(st, wb + 3), wE = P::weight(st, wb + 4),
                      wN = P::weight(st, wb + 6);
  pdl_wait();  // the vectors after the previous kernel in the stream (group.cuh)

  // Step k reads row r_k = t.y - 1 + k (k = 0 .. steps-1) and writes row
  // r_{k-1} (k >= 2).  Row r holds n + 1 - r points, so column c lies inside
  // row r_k exactly for k < n + 2 - t.y - c: one compare of the step index per
  // column.  A point (c, r) is interior when c < len(r) - 1 = len(r + 1), so
  // the row written at step k holds column c as an interior point exactly when
  // the row read at step k holds column c: the write predicate is the read
  // predicate of the same step.
  const int steps = t.z - t.y + 2;
  const int ka = n + 2 - t.y - ca, kb = ka - 1;  // steps whose row holds column ca / cb
  const bool wa = lane >= 1, wbb = lane <= 30;   // lane 0's A and lane 31's B are halo
  int off_s = (t.y - 1) * (n + 2) - ((t.y - 1) * t.y) / 2;  // the row being staged
  int len_s = n + 2 - t.y;
  const T* __restrict__ xa = xm + ca;
  const T* __restrict__ ba = SWEEP ? bm + ca : nullptr;
  // fp32: on the rows where a lane's two columns form an aligned pair (the
  // same for every lane of the warp) one 8-byte copy per vector and one
  // store take both (the load/store queue bounds these kernels; in the
  // float-float and native kernels the extra code costs more than it saves)
  constexpr bool kPairs = sizeof(T) == 4;
  auto stage = [&](int slot, int k) {  // row r_k into ring slot `slot`
    if constexpr (kPairs) {
      const T* src = xa + off_s;
      const T* bsrc = SWEEP ? ba + off_s : src;
      if (k < kb && pair_aligned(reinterpret_cast<const float*>(src)) &&
          pair_aligned(reinterpret_cast<const float*>(bsrc))) {
        cp_async(&ring[slot][lane][0], src, 2 * sizeof(T));
        if (SWEEP) cp_async(&ringb[slot][lane][0], bsrc, 2 * sizeof(T));
        off_s += len_s;
        len_s -= 1;
        return;
      }
    }
    if (k < ka) {
      cp_async(&ring[slot][lane][0], xa + off_s, sizeof(T));
      if (SWEEP) cp_async(&ringb[slot][lane][0], ba + off_s, sizeof(T));
    }
    if (k < kb) {
      cp_async(&ring[slot][lane][1], xa + off_s + 1, sizeof(T));
      if (SWEEP) cp_async(&ringb[slot][lane][1], ba + off_s + 1, sizeof(T));
    }
    off_s += len_s;
    len_s -= 1;
  };
  if constexpr (P::kPoison) {
    // The float-float row marks see every lane's arithmetic, also on columns
    // beyond a row's end, which the ring leaves holding an earlier row's
    // value: the ring starts zeroed (zero-filling copies that read nothing,
    // completed before the first row is staged), so a stale value is zero or
    // an input already split in an earlier row.
#pragma unroll
    for (int k = 0; k < RING; ++k) {
      cp_async_zero(&ring[k][lane][0], xm);
      cp_async_zero(&ring[k][lane][1], xm);
    }
    cp_async_commit();
    cp_async_wait<0>();
  }
#pragma unroll
  for (int k = 0; k < RING; ++k) {
    if (k < steps) stage(k, k);
    cp_async_commit();
  }
  // Columns beyond a row's end hold stale values, which reach only results
  // that are not written.
  // take(k, slot): the row of step k from its ring slot; the slot is then
  // staged again with the row of step k + RING (always in the main walk
  // below, where that step exists; when it does in the tail)
  auto take_g = [&](int k, auto slot_c, auto always_c) -> Row<P> {
    constexpr int slot = decltype(slot_c)::value;
    constexpr bool always = decltype(always_c)::value;
    cp_async_wait<RING - 1>();
    const T va = ring[slot][lane][0], vb = ring[slot][lane][1];
    Row<P> r = make_row<P>(P::conv(va), P::conv(vb));
    if (SWEEP) {  // read before the slot is staged again
      r.b[0] = ringb[slot][lane][0];
      r.b[1] = ringb[slot][lane][1];
    }
    // the slot of step k is free again: stage step k + RING
    if (always || k + RING < steps) stage(slot, k + RING);
    cp_async_commit();
    return r;
  };
  using Always = std::integral_constant<bool, true>;
  using Guarded = std::integral_constant<bool, false>;
  auto take = [&](int k, auto slot_c) -> Row<P> { return take_g(k, slot_c, Guarded{}); };
  int off_o = t.y * (n + 2) - (t.y * (t.y + 1)) / 2;  // the row being written
  int len_o = n + 1 - t.y;
  T* __restrict__ ya = ym + ca;
  typename P::Mark mk = P::mark0();
  // output row r_{k-1} from (below, centre, above) = rows r_{k-2}, r_{k-1}, r_k
  auto step = [&](const Row<P>& lo, const Row<P>& ce, const Row<P>& hi, int k) {
    // the interior stencil is symmetric (w(d) = w(-d), made bitwise equal on
    // the host): add opposite neighbours first
    typename P::Acc a;
    P::first(a, wC, ce.v);
    P::add_sym(a, wE, ce.e, ce.w);
    P::add_sym(a, wN, hi.v, lo.v);
    P::add_sym(a, wSE, lo.e, hi.w);
    T outa, outb;
    P::finish(a, outa, outb);
    P::mark(mk, a);  // float-float: notes a row that read an input outside the range
    if (SWEEP) {  // the centre values of the row are u (fp32 data)
      float ua = 0.0f, ub = 0.0f;
      if constexpr (SWEEP) {
        ua = ce.v.x;
        ub = ce.v.y;
      }
      outa = mode_out_staged<MODE, T>(outa, (T)ua, ce.b[0], dint, md.omega);
      outb = mode_out_staged<MODE, T>(outb, (T)ub, ce.b[1], dint, md.omega);
    }
    if constexpr (kPairs) {
      T* dst = ya + off_o;
      if (wa && wbb && k < kb && pair_aligned(reinterpret_cast<const float*>(dst))) {
        *reinterpret_cast<float2*>(dst) = make_float2((float)outa, (float)outb);
      } else {
        if (wa && k < ka) dst[0] = outa;
        if (wbb && k < kb) dst[1] = outb;
      }
    } else {
      if (wa && k < ka) ya[off_o] = outa;
      if (wbb && k < kb) ya[off_o + 1] = outb;
    }
    off_o += len_o;
    len_o -= 1;
  };
  // three rows in registers whose roles rotate, unrolled by three so that no
  // row is ever copied between registers and every ring slot is a constant
  using S0 = std::integral_constant<int, 0>;
  using S1 = std::integral_constant<int, 1>;
  using S2 = std::integral_constant<int, 2>;
  Row<P> r0 = take(0, S0{});
  Row<P> r1 = take(1, S1{});
  Row<P> r2;
  int k = 2;
  // main walk: all three steps of a pass exist and stage a later row, so the
  // pass has no branch inside (the code generator may interleave the split
  // of one row with the arithmetic of the previous one)
  for (; k + 2 + RING < steps; k += 3) {
    r2 = take_g(k, S2{}, Always{});
    step(r0, r1, r2, k);
    r0 = take_g(k + 1, S0{}, Always{});
    step(r1, r2, r0, k + 1);
    r1 = take_g(k + 2, S1{}, Always{});
    step(r2, r0, r1, k + 2);
  }
  // the last steps (at most RING + 2)
  for (; k < steps; k += 3) {
    r2 = take(k, S2{});
    step(r0, r1, r2, k);
    if (k + 1 >= steps) break;
    r0 = take(k + 1, S0{});
    step(r1, r2, r0, k + 1);
    if (k + 2 >= steps) break;
    r1 = take(k + 2, S1{});
    step(r2, r0, r1, k + 2);
  }
  cp_async_wait<0>();
  if constexpr (P::kPoison) {
    // a row of this lane read an input outside the float-float range: its
    // two columns of the tile again, in native fp64 from memory
    if (P::marked(mk)) {
      const double* wd = st.d + wb;
      Cursor rw;
      rw.init(n, t.y);
      for (int r = t.y; r < t.z; ++r) {
        if (wa && ca < rw.len - 1) ym[rw.off + ca] = native_row2d(xm + rw.off + ca, rw.len, wd);
        if (wbb && cb < rw.len - 1) ym[rw.off + cb] = native_row2d(xm + rw.off + cb, rw.len, wd);
        rw.next();
      }
    }
  }
}

// Blocks per SM the kernel is built for: three for float-float (80
// registers), the compiler's own choice otherwise.
template <class P>
struct MinBlocks2 {
  static constexpr int value = P::kPoison ? 3 : 0;
};

template <class P, int MODE>
__global__ void __launch_bounds__(Thr2<MODE>::value, MinBlocks2<P>::value) k_interior2d(const typename P::T* __restrict__ x,
                                                          typename P::T* __restrict__ y,
                                                          const int4* __restrict__ tiles, int n_tiles,
                                                          int64_t n_warps, int64_t S, int n, StencilPtr st,
                                                          const int4* __restrict__ items, int n_items,
                                                          const Prim* __restrict__ prims,
                                                          const Inc* __restrict__ incs, int n_if_blocks,
                                                          ModeArgs md) {
  using T = typename P::T;
  constexpr int THR = Thr2<MODE>::value;
  constexpr bool SWEEP = MODE == MODE_JACOBI || MODE == MODE_RESIDUAL;
  __shared__ __align__(8) T ring_all[THR / 32][RING][32][2];
  __shared__ __align__(8) T ringb_all[SWEEP ? THR / 32 : 1][RING][32][2];
  pdl_trigger();
  apply2d_block<P, MODE>((int)blockIdx.x, x, y, tiles, n_tiles, n_warps, S, n, st, items, n_items, prims, incs,
                         n_if_blocks, md, ring_all, ringb_all);
}

// ---- batched apply: many meshes in one launch ------------------------------------
// Each mesh of the batch owns a consecutive range of the launch's blocks (its
// interface blocks, then its tile blocks, exactly as in its own launch); a
// block finds its mesh by binary search over the ranges.  The descriptors
// travel as a kernel parameter, so the launch allocates nothing.
struct Apply2dDesc {
  const void* x;
  void* y;
  const int4* tiles;
  const int4* items;
  const Prim* prims;
  const Inc* incs;
  StencilPtr st;
  ModeArgs md;  // the sweep modes' b, inverse diagonal and omega
  int64_t n_warps;
  int64_t S;
  int n_tiles, n, n_items, n_if_blocks;
  int block_begin;  // first block of this mesh in the launch
};
constexpr int BATCH2D = 64;  // meshes per launch (the parameter block stays below 10 KB)
struct Apply2dBatch {
  Apply2dDesc d[BATCH2D];
  int count;
};

template <class P, int MODE>
__global__ void __launch_bounds__(Thr2<MODE>::value, MinBlocks2<P>::value) k_interior2d_batch(const __grid_constant__ Apply2dBatch b) {
  using T = typename P::T;
  constexpr int THR = Thr2<MODE>::value;
  constexpr bool SWEEP = MODE == MODE_JACOBI || MODE == MODE_RESIDUAL;
  __shared__ __align__(8) T ring_all[THR / 32][RING][32][2];
  __shared__ __align__(8) T ringb_all[SWEEP ? THR / 32 : 1][RING][32][2];
  pdl_trigger();
  int lo = 0, hi = b.count - 1;  // the last mesh whose range starts at or before this block
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.d[mid].block_begin <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const Apply2dDesc& d = b.d[lo];
  apply2d_block<P, MODE>((int)blockIdx.x - d.block_begin, static_cast<const T*>(d.x), static_cast<T*>(d.y), d.tiles,
                         d.n_tiles > 0 ? d.n_tiles : 1, d.n_warps, d.S, d.n, d.st, d.items, d.n_items, d.prims,
                         d.incs, d.n_if_blocks, d.md, ring_all, ringb_all);
}

// Element-type index of a policy (1 float-float, 2 fp32, 3 native fp64).
template <class P>
constexpr int dt_of() {
  return sizeof(typename P::T) == 4 ? 2 : (P::kPoison ? 1 : 3);
}

// The tile list of a level for a policy: the autotuned one when present,
// else the default list of its element size.
template <class P>
__host__ void tiles_of(const LevelDev& L, const int4** tiles, int* n_tiles) {
  constexpr int dt = dt_of<P>();
  if (L.tiles_dt[dt]) {
    *tiles = L.tiles_dt[dt];
    *n_tiles = L.n_tiles_dt[dt];
  } else {
    const bool f32 = dt == 2;
    *tiles = f32 ? L.tiles32 : L.tiles;
    *n_tiles = f32 ? L.n_tiles32 : L.n_tiles;
  }
}

template <class P, int MODE>
cudaError_t launch_on(const Mesh& m, const LevelDev& L, const int4* tiles, int n_tiles, const void* x, void* y,
                      cudaStream_t s, const ModeArgs& md) {
  const int64_t n_warps = (int64_t)n_tiles * m.n_cells;
  const int threads = Thr2<MODE>::value;
  const int64_t int_blocks = (n_warps * 32 + threads - 1) / threads;
  const int per = threads / 128;  // interface items per block
  const int if_blocks = (L.n_items + per - 1) / per;
  if (int_blocks + if_blocks == 0) return cudaSuccess;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  return launch_pdl(k_interior2d<P, MODE>, dim3((unsigned)(int_blocks + if_blocks)), dim3(threads), 0, s,
                    (const typename P::T*)x, (typename P::T*)y, tiles, n_tiles > 0 ? n_tiles : 1, n_warps,
                    L.slots_per_macro, L.n, st, (const int4*)L.items, L.n_items, (const Prim*)m.d_prims,
                    (const Inc*)m.d_incs, if_blocks, md);
}

template <class P, int MODE>
cudaError_t launch(const Mesh& m, const LevelDev& L, const void* x, void* y, cudaStream_t s, const ModeArgs& md) {
  const int4* tiles = nullptr;
  int n_tiles = 0;
  tiles_of<P>(L, &tiles, &n_tiles);
  return launch_on<P, MODE>(m, L, tiles, n_tiles, x, y, s, md);
}

template <class P, int MODE = MODE_APPLY>
cudaError_t launch_batch_t(const Mesh* const* meshes, const int* levels, const void* const* xs, void* const* ys,
                           int count, cudaStream_t s, const ModeArgs* mds = nullptr) {
  constexpr int THR = Thr2<MODE>::value;
  Apply2dBatch b;
  for (int i0 = 0; i0 < count; i0 += BATCH2D) {
    b.count = 0;
    int blocks = 0;
    for (int i = i0; i < count && i < i0 + BATCH2D; ++i) {
      const Mesh& m = *meshes[i];
      const LevelDev& L = m.levels[levels[i]];
      const int4* tiles = nullptr;
      int n_tiles = 0;
      tiles_of<P>(L, &tiles, &n_tiles);
      const int64_t n_warps = (int64_t)n_tiles * m.n_cells;
      const int64_t int_blocks = (n_warps * 32 + THR - 1) / THR;
      const int if_blocks = (L.n_items + THR / 128 - 1) / (THR / 128);
      if (int_blocks + if_blocks == 0) continue;
      if ((int64_t)blocks + int_blocks + if_blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
      Apply2dDesc& d = b.d[b.count++];
      d.x = xs[i];
      d.y = ys[i];
      d.tiles = tiles;
      d.items = L.items;
      d.prims = m.d_prims;
      d.incs = m.d_incs;
      d.st = StencilPtr{L.st64, L.st32, L.st_hi, L.st_lo};
      d.md = mds ? mds[i] : ModeArgs{nullptr, nullptr, 0.0};
      d.n_warps = n_warps;
      d.S = L.slots_per_macro;
      d.n_tiles = n_tiles;
      d.n = L.n;
      d.n_items = L.n_items;
      d.n_if_blocks = if_blocks;
      d.block_begin = blocks;
      blocks += int(int_blocks + if_blocks);
    }
    if (b.count == 0) continue;
    const cudaError_t e = launch_pdl(k_interior2d_batch<P, MODE>, dim3(blocks), dim3(THR), 0, s, b);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_apply2d(int dtype, const Mesh& m, const LevelDev& L, const void* x, void* y, cudaStream_t s) {
  const ModeArgs md{nullptr, nullptr, 0.0};
  switch (dtype) {
    case 1: return launch<ArF64FF, MODE_APPLY>(m, L, x, y, s, md);
    case 2: return launch<ArF32, MODE_APPLY>(m, L, x, y, s, md);
    case 3: return launch<ArF64Native, MODE_APPLY>(m, L, x, y, s, md);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_apply2d_partial(int dtype, const Mesh& m, const LevelDev& L, const void* x, void* y,
                                   cudaStream_t s) {
  const ModeArgs md{nullptr, nullptr, 0.0};
  switch (dtype) {
    case 1: return launch<ArF64FF, MODE_PARTIAL>(m, L, x, y, s, md);
    case 2: return launch<ArF32, MODE_PARTIAL>(m, L, x, y, s, md);
    case 3: return launch<ArF64Native, MODE_PARTIAL>(m, L, x, y, s, md);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_apply2d_tiles(int dtype, const Mesh& m, const LevelDev& L, const int4* tiles, int n_tiles,
                                 const void* x, void* y, cudaStream_t s) {
  const ModeArgs md{nullptr, nullptr, 0.0};
  switch (dtype) {
    case 1: return launch_on<ArF64FF, MODE_APPLY>(m, L, tiles, n_tiles, x, y, s, md);
    case 2: return launch_on<ArF32, MODE_APPLY>(m, L, tiles, n_tiles, x, y, s, md);
    case 3: return launch_on<ArF64Native, MODE_APPLY>(m, L, tiles, n_tiles, x, y, s, md);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep2d(int dtype, bool jacobi, const Mesh& m, const LevelDev& L, const void* u, const void* b,
                           const void* dinv, double omega, void* out, cudaStream_t s) {
  const ModeArgs md{b, dinv, omega};
  switch (dtype) {
    case 2:
      return jacobi ? launch<ArF32, MODE_JACOBI>(m, L, u, out, s, md) : launch<ArF32, MODE_RESIDUAL>(m, L, u, out, s, md);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sweep2d_group(bool jacobi, const Mesh* const* ms, const int* levels, const void* const* u,
                                 const void* const* b, const void* const* dinv, const double* omega,
                                 void* const* out, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  std::vector<ModeArgs> md(count);
  for (int i = 0; i < count; ++i) md[i] = ModeArgs{b[i], dinv[i], omega[i]};
  return jacobi ? launch_batch_t<ArF32, MODE_JACOBI>(ms, levels, u, out, count, s, md.data())
                : launch_batch_t<ArF32, MODE_RESIDUAL>(ms, levels, u, out, count, s, md.data());
}

cudaError_t launch_apply2d_batch(int dtype, const Mesh* const* meshes, const int* levels, const void* const* xs,
                                 void* const* ys, int count, cudaStream_t s) {
  switch (dtype) {
    case 1: return launch_batch_t<ArF64FF>(meshes, levels, xs, ys, count, s);
    case 2: return launch_batch_t<ArF32>(meshes, levels, xs, ys, count, s);
    case 3: return launch_batch_t<ArF64Native>(meshes, levels, xs, ys, count, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
