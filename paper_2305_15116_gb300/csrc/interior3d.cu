// Macro-interior stencil sweep, 3D: the 15-point stencil of a refined
// macro-tetrahedron (the 3D extension the paper names as its next step,
// Sec. 6).  The refinement inside a macro is the Kuhn/Freudenthal one, whose
// edges give the offsets
//   0, ±(1,0,0), ±(0,1,0), ±(0,0,1), ±(1,-1,0), ±(1,0,-1), ±(0,1,-1), ±(1,-1,1).
// A macro array stacks triangular slices along z; slice z has side n+1-z and
// starts at T3(n+1) - T3(n+1-z), T3(k) = k(k+1)(k+2)/6; inside a slice the
// layout is the 2D one.
//
// GPU mapping: as in 2D, one warp per tile of 32 columns x up to 64 rows of
// one slice z; the warp walks up the rows of slice z and, in step, of the
// slices z+1 and z-1, holding the rows it needs in registers and taking the
// x-neighbours from adjacent lanes by shuffles.
#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

template <class P>
struct Row {
  typename P::V v, w, e;
};

__device__ __forceinline__ int64_t slice_start(int n, int z) {
  const int64_t N = n + 1;
  const int64_t a = N, b = N - z;
  return a * (a + 1) * (a + 2) / 6 - b * (b + 1) * (b + 2) / 6;
}

template <class P>
__device__ __forceinline__ Row<P> load_row(const typename P::T* __restrict__ xm, int n, int z, int64_t zs,
                                           int r, int col) {
  const int64_t side = n + 1 - z;
  const int64_t start = zs + (int64_t)r * side - ((int64_t)r * (r - 1)) / 2;
  typename P::V v = (col <= n - z - r) ? P::load(xm + start + col) : P::zero();
  return Row<P>{v, P::up(v), P::down(v)};
}

template <class P>
__global__ void __launch_bounds__(256) k_interior3d(const typename P::T* __restrict__ x,
                                                    typename P::T* __restrict__ y,
                                                    const int4* __restrict__ tiles, int n_tiles,
                                                    int64_t n_warps, int64_t S, int n, StencilPtr st) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;
  const int lane = threadIdx.x & 31;
  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];
  const int z = t.w;
  const int col = t.x - 1 + lane;
  const typename P::T* __restrict__ xm = x + m * S;
  typename P::T* __restrict__ ym = y + m * S;

  const int64_t wb = m * (int64_t)(NCLS3 * NW3);
  typename P::W w[NW3];
#pragma unroll
  for (int k = 0; k < NW3; ++k) w[k] = P::weight(st, wb + k);

  const int64_t z0 = slice_start(n, z), zu = slice_start(n, z + 1), zd = slice_start(n, z - 1);
  Row<P> prev = load_row<P>(xm, n, z, z0, t.y - 1, col);
  Row<P> cur = load_row<P>(xm, n, z, z0, t.y, col);
  Row<P> uprev = load_row<P>(xm, n, z + 1, zu, t.y - 1, col);
  Row<P> dcur = load_row<P>(xm, n, z - 1, zd, t.y, col);
  const bool writer = lane >= 1 && lane <= 30;
  const int64_t side = n + 1 - z;
  for (int r = t.y; r < t.z; ++r) {
    const Row<P> nxt = load_row<P>(xm, n, z, z0, r + 1, col);
    const Row<P> ucur = load_row<P>(xm, n, z + 1, zu, r, col);
    const Row<P> dnxt = load_row<P>(xm, n, z - 1, zd, r + 1, col);
    typename P::Acc1 a;
    P::first1(a, w[0], cur.v);
    P::add1(a, w[1], cur.e);     // ( 1, 0, 0)
    P::add1(a, w[2], cur.w);     // (-1, 0, 0)
    P::add1(a, w[3], nxt.v);     // ( 0, 1, 0)
    P::add1(a, w[4], prev.v);    // ( 0,-1, 0)
    P::add1(a, w[5], prev.e);    // ( 1,-1, 0)
    P::add1(a, w[6], nxt.w);     // (-1, 1, 0)
    P::add1(a, w[7], ucur.v);    // ( 0, 0, 1)
    P::add1(a, w[8], ucur.w);    // (-1, 0, 1)
    P::add1(a, w[9], uprev.v);   // ( 0,-1, 1)
    P::add1(a, w[10], uprev.e);  // ( 1,-1, 1)
    P::add1(a, w[11], dcur.v);   // ( 0, 0,-1)
    P::add1(a, w[12], dcur.e);   // ( 1, 0,-1)
    P::add1(a, w[13], dnxt.v);   // ( 0, 1,-1)
    P::add1(a, w[14], dnxt.w);   // (-1, 1,-1)
    if (writer && col <= n - 1 - z - r) {
      const int64_t start = z0 + (int64_t)r * side - ((int64_t)r * (r - 1)) / 2;
      ym[start + col] = P::finish1(a);
    }
    prev = cur;
    cur = nxt;
    uprev = ucur;
    dcur = dnxt;
  }
}

template <class P>
cudaError_t launch(const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s) {
  if (L.n_tiles == 0) return cudaSuccess;
  const int64_t n_warps = (int64_t)L.n_tiles * n_cells;
  const int threads = 256;
  const int64_t blocks = (n_warps * 32 + threads - 1) / threads;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  k_interior3d<P><<<(unsigned)blocks, threads, 0, s>>>((const typename P::T*)x, (typename P::T*)y, L.tiles,
                                                       L.n_tiles, n_warps, L.slots_per_macro, L.n, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interior3d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y,
                              cudaStream_t s) {
  switch (dtype) {
    case 1: return launch<ArF64FF>(L, n_cells, x, y, s);
    case 2: return launch<ArF32>(L, n_cells, x, y, s);
    case 3: return launch<ArF64Native>(L, n_cells, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
