// Macro-interior stencil sweep, 2D (the vertex-to-vertex kernel of Sec. 4.2).
//
// For every macro-triangle m and every point strictly inside it
// (x >= 1, y >= 1, x + y <= n - 1):
//   y[x,y] = C x[x,y] + E x[x+1,y] + W x[x-1,y] + N x[x,y+1] + S x[x,y-1]
//          + SE x[x+1,y-1] + NW x[x-1,y+1]
// with the constant weights of macro m.  The triangular array of a macro is
// row-major with x contiguous; row r starts at r(n+2) - r(r+1)/2 (Sec. 3).
//
// GPU mapping: one warp per tile of 32 consecutive columns and up to 64 rows.
// Each lane owns one column and walks up the rows, keeping three rows in
// registers (the layer condition of Sec. 2.3 held in the register file); the
// left/right neighbours come from the adjacent lanes by warp shuffles, so
// every value is read from memory once per tile plus the two halo rows.  The
// 30 inner lanes write; lanes 0 and 31 only supply the horizontal halo.
#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

template <class P>
struct Row {
  typename P::V v, w, e;  // value of this lane's column, of column-1, of column+1
};

template <class P>
__device__ __forceinline__ Row<P> load_row(const typename P::T* __restrict__ xm, int n, int r, int col) {
  const int64_t start = (int64_t)r * (n + 2) - ((int64_t)r * (r + 1)) / 2;
  typename P::V v = (col <= n - r) ? P::load(xm + start + col) : P::zero();
  return Row<P>{v, P::up(v), P::down(v)};
}

template <class P>
__global__ void __launch_bounds__(256) k_interior2d(const typename P::T* __restrict__ x,
                                                    typename P::T* __restrict__ y,
                                                    const int4* __restrict__ tiles, int n_tiles,
                                                    int64_t n_warps, int64_t S, int n, StencilPtr st) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];
  const int col = t.x - 1 + lane;
  const typename P::T* __restrict__ xm = x + m * S;
  typename P::T* __restrict__ ym = y + m * S;

  const int64_t wb = m * (int64_t)(NCLS2 * NW2);  // class 0: the full interior stencil
  const typename P::Wt wS = P::weight(st, wb + 0), wSE = P::weight(st, wb + 1), wW = P::weight(st, wb + 2),
                       wC = P::weight(st, wb + 3), wE = P::weight(st, wb + 4), wNW = P::weight(st, wb + 5),
                       wN = P::weight(st, wb + 6);

  Row<P> prev = load_row<P>(xm, n, t.y - 1, col);
  Row<P> cur = load_row<P>(xm, n, t.y, col);
  const bool writer = lane >= 1 && lane <= 30;
#pragma unroll 2
  for (int r = t.y; r < t.z; ++r) {
    const Row<P> nxt = load_row<P>(xm, n, r + 1, col);
    typename P::Acc a;
    P::first(a, wC, cur.v);
    P::add(a, wE, cur.e);
    P::add(a, wW, cur.w);
    P::add(a, wN, nxt.v);
    P::add(a, wS, prev.v);
    P::add(a, wSE, prev.e);
    P::add(a, wNW, nxt.w);
    if (writer && col <= n - 1 - r) {
      const int64_t start = (int64_t)r * (n + 2) - ((int64_t)r * (r + 1)) / 2;
      ym[start + col] = P::finish(a);
    }
    prev = cur;
    cur = nxt;
  }
}

template <class P>
cudaError_t launch(const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  const int64_t n_warps = (int64_t)L.n_tiles * n_cells;
  const int threads = 256;
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
