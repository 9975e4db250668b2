// Macro-interior stencil sweep, 2D (the vertex-to-vertex kernel of Sec. 4.2).
//
// For every macro-triangle m and every point strictly inside it
// (x >= 1, y >= 1, x + y <= n - 1):
//   y[x,y] = C x[x,y] + E x[x+1,y] + W x[x-1,y] + N x[x,y+1] + S x[x,y-1]
//          + SE x[x+1,y-1] + NW x[x-1,y+1]
// with the constant weights of macro m.  The triangular array of a macro is
// row-major with x contiguous; row r starts at r(n+2) - r(r+1)/2 and holds
// n+1-r points (Sec. 3).
//
// GPU mapping: one warp per tile of 32 consecutive columns and up to 64 rows.
// The tile's rows are split into two halves that the warp walks up in
// lockstep ("streams" A and B), so every lane evaluates two independent
// points per step and the float-float arithmetic runs on packed f32x2
// instructions.  Each lane stages its column of the next RING rows of both
// streams in shared memory with cp.async, which keeps 2 x RING loads per warp
// in flight without spending registers on them.  Each lane owns one column and
// keeps three rows per stream in registers (the layer condition of Sec. 2.3
// held in the register file); left/right neighbours come from the adjacent
// lanes by warp shuffles, so every value is read from memory once per stream
// plus two halo rows.  The 30 inner lanes write; lanes 0 and 31 only supply
// the horizontal halo.
#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

template <class P>
struct Row {
  typename P::V v, w, e;  // value of this lane's column, of column-1, of column+1
};

template <class P>
__device__ __forceinline__ Row<P> make_row(typename P::V v) {
  return Row<P>{v, P::up(v), P::down(v)};
}

// Row-walking cursor: offset of row r inside the macro array and its length.
struct Cursor {
  int off;  // r(n+2) - r(r+1)/2
  int len;  // n + 1 - r
  int r;
  __device__ __forceinline__ void init(int n, int row) {
    r = row;
    off = row * (n + 2) - (row * (row + 1)) / 2;
    len = n + 1 - row;
  }
  __device__ __forceinline__ void next() {
    off += len;
    len -= 1;
    r += 1;
  }
};

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows in flight per stream: each lane stages its own column of the next RING
// rows of both streams in shared memory with cp.async, so a warp keeps
// 2 x RING loads outstanding without holding them in registers.
constexpr int RING = 8;
constexpr int THREADS2D = 256;

template <class P>
__global__ void __launch_bounds__(THREADS2D) k_interior2d(const typename P::T* __restrict__ x,
                                                          typename P::T* __restrict__ y,
                                                          const int4* __restrict__ tiles, int n_tiles,
                                                          int64_t n_warps, int64_t S, int n, StencilPtr st) {
  using T = typename P::T;
  __shared__ T ring_all[THREADS2D / 32][2][RING][32];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  T(*ring)[RING][32] = ring_all[threadIdx.x >> 5];
  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];
  const int col = t.x - 1 + lane;
  const T* __restrict__ xm = x + m * S;
  T* __restrict__ ym = y + m * S;

  const int64_t wb = m * (int64_t)(NCLS2 * NW2);  // class 0: the full interior stencil
  const typename P::W wS = P::weight(st, wb + 0), wSE = P::weight(st, wb + 1), wW = P::weight(st, wb + 2),
                      wC = P::weight(st, wb + 3), wE = P::weight(st, wb + 4), wNW = P::weight(st, wb + 5),
                      wN = P::weight(st, wb + 6);

  // stream A writes rows [t.y, t.y + h), stream B rows [t.y + h, t.z); each
  // stream reads rows from one below its first to one above its last output
  const int h = (t.z - t.y + 1) >> 1;
  const int nb = t.z - t.y - h;  // nb == h or h - 1
  const int steps = h + 2;       // rows read per stream
  Cursor ia, ib;                 // next row to stage, per stream
  ia.init(n, t.y - 1);
  ib.init(n, t.y + h - 1);
  // prologue: stage rows 0 .. RING-1 of both streams
#pragma unroll
  for (int k = 0; k < RING; ++k) {
    if (k < steps) {
      if (col < ia.len) cp_async(&ring[0][k][lane], xm + ia.off + col, sizeof(T));
      if (col < ib.len) cp_async(&ring[1][k][lane], xm + ib.off + col, sizeof(T));
      ia.next();
      ib.next();
    }
    cp_async_commit();
  }
  Cursor ca, cb;  // row being consumed, per stream
  ca.init(n, t.y - 1);
  cb.init(n, t.y + h - 1);
  auto take = [&](int k, int s, const Cursor& c) -> typename P::V {
    // value of this lane's column in the row consumed at step k of stream s
    const T v = ring[s][k % RING][lane];
    return (col < c.len) ? P::conv(v) : P::zero();
  };
  auto refill = [&](int k) {
    // the slot of step k is free again: stage step k + RING
    if (k + RING < steps) {
      if (col < ia.len) cp_async(&ring[0][k % RING][lane], xm + ia.off + col, sizeof(T));
      if (col < ib.len) cp_async(&ring[1][k % RING][lane], xm + ib.off + col, sizeof(T));
      ia.next();
      ib.next();
    }
    cp_async_commit();
  };
  cp_async_wait<RING - 1>();
  Row<P> pa = make_row<P>(take(0, 0, ca));
  Row<P> pb = make_row<P>(take(0, 1, cb));
  refill(0);
  ca.next();
  cb.next();
  cp_async_wait<RING - 1>();
  Row<P> qa = make_row<P>(take(1, 0, ca));
  Row<P> qb = make_row<P>(take(1, 1, cb));
  refill(1);
  const bool writer = lane >= 1 && lane <= 30;
  for (int i = 0; i < h; ++i) {
    // ca / cb point at the rows being written; read the rows above them
    Cursor na = ca, nbc = cb;
    na.next();
    nbc.next();
    cp_async_wait<RING - 1>();
    const Row<P> ra = make_row<P>(take(i + 2, 0, na));
    const Row<P> rb = make_row<P>(take(i + 2, 1, nbc));
    refill(i + 2);
    typename P::Acc a;
    P::first(a, wC, P::pair(qa.v, qb.v));
    P::add(a, wE, P::pair(qa.e, qb.e));
    P::add(a, wW, P::pair(qa.w, qb.w));
    P::add(a, wN, P::pair(ra.v, rb.v));
    P::add(a, wS, P::pair(pa.v, pb.v));
    P::add(a, wSE, P::pair(pa.e, pb.e));
    P::add(a, wNW, P::pair(ra.w, rb.w));
    typename P::T outa, outb;
    P::finish(a, outa, outb);
    // point (col, r) is interior when col <= n - 1 - r, i.e. col < len - 1
    if (writer && col < ca.len - 1) ym[ca.off + col] = outa;
    if (writer && i < nb && col < cb.len - 1) ym[cb.off + col] = outb;
    pa = qa;
    qa = ra;
    pb = qb;
    qb = rb;
    ca = na;
    cb = nbc;
  }
  cp_async_wait<0>();
}

template <class P>
cudaError_t launch(const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  const int64_t n_warps = (int64_t)L.n_tiles * n_cells;
  const int threads = THREADS2D;
  const int64_t blocks = (n_warps * 32 + threads - 1) / threads;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  k_interior2d<P><<<(unsigned)blocks, threads, 0, s>>>((const typename P::T*)x, (typename P::T*)y, L.tiles,
                                                       L.n_tiles, n_warps, L.slots_per_macro, L.n, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interior2d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y,
                              cudaStream_t s) {
  switch (dtype) {
    case 1: return launch<ArF64FF>(L, n_cells, x, y, s);
    case 2: return launch<ArF32>(L, n_cells, x, y, s);
    case 3: return launch<ArF64Native>(L, n_cells, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
