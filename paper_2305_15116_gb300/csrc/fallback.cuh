// Native fp64 rows for the float-float kernels.
//
// A float-float kernel whose row read an input outside the float-float range
// (arith.cuh) recomputes that row here, in native fp64 FMA arithmetic,
// straight from the float64 vector in global memory: the same weights (the
// fp64 class table), the same neighbours.  Taken only for such rows, so
// these functions favour few registers over speed.
#pragma once

#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

// 2D macro-interior row of the point at p (row length len = n + 1 - y):
// weights w[0..6] in the order S, SE, W, C, E, NW, N.  Row y+1 starts len
// slots after row y, row y-1 len + 1 slots before it.
__device__ __forceinline__ double native_row2d(const double* __restrict__ p, int len,
                                                   const double* __restrict__ w) {
  double a = __dmul_rn(__ldg(w + 3), __ldg(p));
  a = __fma_rn(__ldg(w + 4), __ldg(p + 1), a);
  a = __fma_rn(__ldg(w + 2), __ldg(p - 1), a);
  a = __fma_rn(__ldg(w + 6), __ldg(p + len), a);
  a = __fma_rn(__ldg(w + 5), __ldg(p + len - 1), a);
  a = __fma_rn(__ldg(w + 0), __ldg(p - len - 1), a);
  a = __fma_rn(__ldg(w + 1), __ldg(p - len), a);
  return a;
}

// Slot of lattice point (x, y, z) inside a 3D macro array of level n = 2^L.
__device__ __forceinline__ int64_t fb_slot3(int n, int x, int y, int z) {
  const int64_t N = n + 1, b = N - z;
  return N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6 + (int64_t)y * b - ((int64_t)y * (y - 1)) / 2 + x;
}

// 3D row of point (px, py, pz) of the macro array xm with the 15 weights w
// (centre, the six in-slice neighbours, four of slice z+1, four of slice z-1,
// in the order of the kernels' weight slots).  Neighbours outside the macro
// carry weight 0 in every class stencil and are skipped.
__device__ __forceinline__ double native_row3d(const double* __restrict__ xm, int n, int px, int py, int pz,
                                                   const double* __restrict__ w) {
  const signed char off[NW3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                   {1, -1, 0}, {-1, 1, 0}, {0, 0, 1},  {-1, 0, 1}, {0, -1, 1},
                                   {1, -1, 1}, {0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {-1, 1, -1}};
  double a = 0.0;
  for (int k = 0; k < NW3; ++k) {
    const int qx = px + off[k][0], qy = py + off[k][1], qz = pz + off[k][2];
    if (qx < 0 || qy < 0 || qz < 0 || qx + qy + qz > n) continue;
    const double wk = __ldg(w + k);
    if (wk != 0.0) a = __fma_rn(wk, __ldg(xm + fb_slot3(n, qx, qy, qz)), a);
  }
  return a;
}

}  // namespace hyteg
