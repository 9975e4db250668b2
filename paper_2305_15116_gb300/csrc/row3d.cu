// 3D stencil sweep over every slot of every macro-tetrahedron (the 15-point
// Kuhn stencil; the paper's 3D extension, Sec. 7), as a warp row kernel.
//
// A macro array stacks triangular slices z = 0..n (slice z has side
// M = n+1-z and starts at T3(n+1) - T3(n+1-z), T3(k) = k(k+1)(k+2)/6); the
// stencil of point (x, y, z) reads
//   slice z:   rows y-1, y, y+1  (the 2D 7-point shape),
//   slice z+1: (0,0,1) (-1,0,1) on row y, (0,-1,1) (1,-1,1) on row y-1,
//   slice z-1: (0,0,-1) (1,0,-1) on row y, (0,1,-1) (-1,1,-1) on row y+1.
// One warp takes a tile of 32 lattice columns (30 written) and up to 64 rows
// of one slice of one macro and walks up the rows: cp.async stages the next
// row of slices z-1, z and z+1 for the lane's column, three rows of each stay
// in registers with their x-1 / x+1 neighbours fetched once per row by warp
// shuffles.  Values outside the macro (columns past a row's end, rows past a
// slice's end, slices -1 and n+1) read as zero.
//
// Every slot is written: points inside the macro with the macro's interior
// stencil (symmetric, w(d) = w(-d), so opposite neighbours are added first),
// points on its faces, edges and vertices with the partial stencil of their
// boundary class (only the macro's own micro-tets; its weights are zero where
// a neighbour lies outside the macro, and that neighbour reads as zero).  The
// two ends of every row (x = 0 and x + y + z = n) are left to
// k_row3d_lines, one thread per point, so that the class inside the row
// kernel is the same for all lanes of a row (y = 0 rows and the z = 0 slice
// take their partial stencils uniformly).  The interface step then sums the
// copies' partial rows (k_interface_reduce).
#include "arith.cuh"
#include "fallback.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

// Single-point symmetric product-accumulate acc += w * (u + v), per policy.
template <class P>
struct Sym;
template <>
struct Sym<ArF32> {
  static __device__ __forceinline__ void add(float& a, const ArF32::W& w, float u, float v) {
    a = __fmaf_rn(w, __fadd_rn(u, v), a);
  }
};
template <>
struct Sym<ArF64Native> {
  static __device__ __forceinline__ void add(double& a, const ArF64Native::W& w, double u, double v) {
    a = __fma_rn(w, __dadd_rn(u, v), a);
  }
};
template <>
struct Sym<ArF64FF> {
  // the high parts are added exactly (TwoSum), the low parts and the error
  // form the low part of the pair sum, then one product-accumulate
  static __device__ __forceinline__ void add(ArF64FF::Acc1& a, const ArF64FF::W& w, FF u, FF v) {
    const float sh = __fadd_rn(u.h, v.h);
    const float bb = __fsub_rn(sh, u.h);
    const float er = __fadd_rn(__fsub_rn(u.h, __fsub_rn(sh, bb)), __fsub_rn(v.h, bb));
    const float sl = __fadd_rn(__fadd_rn(u.l, v.l), er);
    ArF64FF::add1(a, w, FF{sh, sl});
  }
};

// One row of the three slices seen from one lane: own value and the x+1 (e)
// and x-1 (w) neighbours.
template <class P>
struct Trip {
  typename P::V c, e, w;
};
template <class P>
struct Rec {
  Trip<P> z, u, d;  // slice z, z+1, z-1
};

template <class P>
__device__ __forceinline__ Trip<P> trip(typename P::V v) {
  return Trip<P>{v, P::down(v), P::up(v)};
}

__device__ __forceinline__ void r3_cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem));
}
// a shared-memory element of `bytes` (4 or 8) set to zero by an asynchronous
// copy that reads no bytes (src, a valid global address, is not accessed)
__device__ __forceinline__ void r3_cp_zero(void* smem, const void* src, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, 0;" ::"r"(sa), "l"(src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, 0;" ::"r"(sa), "l"(src));
}
__device__ __forceinline__ void r3_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void r3_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int R3THREADS = 256;
template <class T>
struct R3Ring {
  static constexpr int value = sizeof(T) == 4 ? 8 : 4;  // rows in flight per warp
};

// Row cursor of one slice: offset and length of row r (32-bit, inside the macro).
struct SCur {
  int off, len;
  __device__ __forceinline__ void init(int n, int z, int r) {
    const int64_t N = n + 1;
    const int M = int(N) - z;  // slice side
    const int zs = int((N * (N + 1) * (N + 2)) / 6 - (int64_t(M) * (M + 1) * (M + 2)) / 6);
    off = zs + r * M - (r * (r - 1)) / 2;
    len = (z < 0 || z > n) ? 0 : M - r;
  }
  __device__ __forceinline__ void next() {
    off += len;
    len -= 1;
  }
};

template <class P>
__global__ void __launch_bounds__(R3THREADS) k_row3d(const typename P::T* __restrict__ x, typename P::T* __restrict__ y,
                                                     const int4* __restrict__ tiles, int n_tiles, int64_t n_warps,
                                                     int64_t S, int n, StencilPtr st) {
  using T = typename P::T;
  using V = typename P::V;
  constexpr int RING = R3Ring<T>::value;
  __shared__ T ring_all[R3THREADS / 32][RING][3][32];
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp >= n_warps) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  T(*ring)[3][32] = ring_all[threadIdx.x >> 5];
  const int64_t m = warp / n_tiles;
  const int4 t = tiles[warp - m * n_tiles];  // (x0, y0, y1, z)
  const int z = t.w;
  const int c = t.x - 1 + lane;
  const T* __restrict__ xm = x + m * S;
  T* __restrict__ ym = y + m * S;

  // interior weights (class 0), symmetric pairs: C, (1,0,0), (0,1,0),
  // (1,-1,0), (0,0,1), (-1,0,1), (0,-1,1), (1,-1,1)
  const int64_t wb = m * (int64_t)(NCLS3 * NW3);
  const typename P::W w0 = P::weight(st, wb + 0), w1 = P::weight(st, wb + 1), w3 = P::weight(st, wb + 3),
                      w5 = P::weight(st, wb + 5), w7 = P::weight(st, wb + 7), w8 = P::weight(st, wb + 8),
                      w9 = P::weight(st, wb + 9), w10 = P::weight(st, wb + 10);

  // rows t.y-1 .. t.z of the three slices are read; rows t.y .. t.z-1 of
  // slice z written
  const int steps = t.z - t.y + 2;
  SCur sz, su, sd;  // next rows to stage
  sz.init(n, z, t.y - 1);
  su.init(n, z + 1, t.y - 1);
  sd.init(n, z - 1, t.y - 1);
  int rs = t.y - 1;
  auto stage = [&](int slot) {
    if (rs >= 0 && c >= 0) {
      if (c < sz.len) r3_cp_async(&ring[slot][0][lane], xm + sz.off + c, sizeof(T));
      if (c < su.len) r3_cp_async(&ring[slot][1][lane], xm + su.off + c, sizeof(T));
      if (c < sd.len) r3_cp_async(&ring[slot][2][lane], xm + sd.off + c, sizeof(T));
    }
    ++rs;
    sz.next();
    su.next();
    sd.next();
  };
  if constexpr (P::kPoison) {
    // Float-float: the ring starts zeroed (copies that read nothing, completed
    // before the first row is staged) and a value outside the macro is not
    // selected away: it is zero or an input of an earlier row, met only by
    // zero class weights, and one outside the float-float range marks the
    // row, which is then recomputed in native fp64.
#pragma unroll
    for (int k = 0; k < RING; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) r3_cp_zero(&ring[k][j][lane], xm, sizeof(T));
    r3_commit();
    r3_wait<0>();
  }
#pragma unroll
  for (int k = 0; k < RING; ++k) {
    if (k < steps) stage(k);
    r3_commit();
  }
  SCur cz, cu, cd;  // rows being consumed
  cz.init(n, z, t.y - 1);
  cu.init(n, z + 1, t.y - 1);
  cd.init(n, z - 1, t.y - 1);
  int rc = t.y - 1;
  auto take = [&](int k) -> Rec<P> {
    r3_wait<RING - 1>();
    const int slot = k & (RING - 1);
    const bool ok = rc >= 0 && c >= 0;
    const V vz = P::kPoison || (ok && c < cz.len) ? P::conv(ring[slot][0][lane]) : P::zero();
    const V vu = P::kPoison || (ok && c < cu.len) ? P::conv(ring[slot][1][lane]) : P::zero();
    const V vd = P::kPoison || (ok && c < cd.len) ? P::conv(ring[slot][2][lane]) : P::zero();
    if (k + RING < steps) stage(slot);
    r3_commit();
    ++rc;
    cz.next();
    cu.next();
    cd.next();
    return Rec<P>{trip<P>(vz), trip<P>(vu), trip<P>(vd)};
  };
  const bool writer = lane >= 1 && lane <= 30;
  SCur co;  // output row of slice z
  co.init(n, z, t.y);
  int yo = t.y;
  // the two ends of every row (x = 0 and x + y + z = n) belong to
  // k_row3d_lines; what is left of a row has one class for the whole warp
  const int cls_z = z == 0 ? 4 : 0;
  auto step = [&](const Rec<P>& lo, const Rec<P>& ce, const Rec<P>& hi) {
    if (writer && c >= 1 && c < co.len - 1) {
      const int cls = (yo == 0 ? 2 : 0) | cls_z;
      typename P::Acc1 a;
      if (cls == 0) {
        P::first1(a, w0, ce.z.c);
        Sym<P>::add(a, w1, ce.z.e, ce.z.w);  // (1,0,0) + (-1,0,0)
        Sym<P>::add(a, w3, hi.z.c, lo.z.c);  // (0,1,0) + (0,-1,0)
        Sym<P>::add(a, w5, lo.z.e, hi.z.w);  // (1,-1,0) + (-1,1,0)
        Sym<P>::add(a, w7, ce.u.c, ce.d.c);  // (0,0,1) + (0,0,-1)
        Sym<P>::add(a, w8, ce.u.w, ce.d.e);  // (-1,0,1) + (1,0,-1)
        Sym<P>::add(a, w9, lo.u.c, hi.d.c);  // (0,-1,1) + (0,1,-1)
        Sym<P>::add(a, w10, lo.u.e, hi.d.w); // (1,-1,1) + (-1,1,-1)
      } else {
        // partial stencil of the class; neighbours outside the macro are zero
        const int64_t cb = wb + cls * NW3;
        P::first1(a, P::weight(st, cb + 0), ce.z.c);
        P::add1(a, P::weight(st, cb + 1), ce.z.e);
        P::add1(a, P::weight(st, cb + 2), ce.z.w);
        P::add1(a, P::weight(st, cb + 3), hi.z.c);
        P::add1(a, P::weight(st, cb + 4), lo.z.c);
        P::add1(a, P::weight(st, cb + 5), lo.z.e);
        P::add1(a, P::weight(st, cb + 6), hi.z.w);
        P::add1(a, P::weight(st, cb + 7), ce.u.c);
        P::add1(a, P::weight(st, cb + 8), ce.u.w);
        P::add1(a, P::weight(st, cb + 9), lo.u.c);
        P::add1(a, P::weight(st, cb + 10), lo.u.e);
        P::add1(a, P::weight(st, cb + 11), ce.d.c);
        P::add1(a, P::weight(st, cb + 12), ce.d.e);
        P::add1(a, P::weight(st, cb + 13), hi.d.c);
        P::add1(a, P::weight(st, cb + 14), hi.d.w);
      }
      T r = P::finish1(a);
      if constexpr (P::kPoison) {  // an input outside the float-float range: native fp64 row
        if (P::bad1(a)) r = native_row3d(xm, n, c, yo, z, st.d + wb + cls * NW3);
      }
      ym[co.off + c] = r;
    }
    ++yo;
    co.next();
  };
  // three records in registers whose roles rotate (unrolled by three)
  Rec<P> r0 = take(0);
  Rec<P> r1 = take(1);
  Rec<P> r2;
  for (int k = 2; k < steps; k += 3) {
    r2 = take(k);
    step(r0, r1, r2);
    if (k + 1 >= steps) break;
    r0 = take(k + 1);
    step(r1, r2, r0);
    if (k + 2 >= steps) break;
    r1 = take(k + 2);
    step(r2, r0, r1);
  }
  r3_wait<0>();
}

__device__ __forceinline__ int64_t r3_slot(int n, int x, int y, int z) {
  const int64_t N = n + 1, b = N - z;
  return N * (N + 1) * (N + 2) / 6 - b * (b + 1) * (b + 2) / 6 + (int64_t)y * b - ((int64_t)y * (y - 1)) / 2 + x;
}

__constant__ int c_r3off[NW3][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                    {1, -1, 0}, {-1, 1, 0}, {0, 0, 1},  {-1, 0, 1}, {0, -1, 1},
                                    {1, -1, 1}, {0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {-1, 1, -1}};

// The ends of every row of every slice: (0, y, z) and (n-y-z, y, z), one
// thread each, with the partial stencil of the point's class; neighbours
// outside the macro have weight 0 and are not read.  Rows are numbered
// slice by slice (slice z holds n+1-z rows); thread 2q+e takes end e of row q.
template <class P>
__global__ void __launch_bounds__(128) k_row3d_lines(const typename P::T* __restrict__ x,
                                                     typename P::T* __restrict__ y, int64_t S, int n, int n_rows,
                                                     StencilPtr st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n_rows) return;
  const int q = i >> 1, e = i & 1;
  // slice z of row q: rows before slice z: z(n+1) - z(z-1)/2 (decode with a
  // float estimate and exact integer fix-ups)
  const float b = 2.0f * (n + 1) + 1.0f;
  int z = (int)((b - sqrtf(fmaxf(b * b - 8.0f * q, 0.0f))) * 0.5f);
  z = max(z, 0);
  while (z > 0 && z * (n + 1) - (z * (z - 1)) / 2 > q) --z;
  while ((z + 1) * (n + 1) - ((z + 1) * z) / 2 <= q) ++z;
  const int yy = q - (z * (n + 1) - (z * (z - 1)) / 2);
  const int xend = n - yy - z;
  if (e == 1 && xend == 0) return;  // a one-point row has one end
  const int px = e == 0 ? 0 : xend;
  const int64_t cell = blockIdx.y;
  const typename P::T* __restrict__ xm = x + cell * S;
  const int cls = (px == 0 ? 1 : 0) | (yy == 0 ? 2 : 0) | (z == 0 ? 4 : 0) | (px + yy + z == n ? 8 : 0);
  const int64_t cb = cell * (int64_t)(NCLS3 * NW3) + cls * NW3;
  typename P::Acc1 a;
  P::first1(a, P::weight(st, cb), P::load(xm + r3_slot(n, px, yy, z)));
#pragma unroll
  for (int k = 1; k < NW3; ++k) {
    const int qx = px + c_r3off[k][0], qy = yy + c_r3off[k][1], qz = z + c_r3off[k][2];
    if (qx < 0 || qy < 0 || qz < 0 || qx + qy + qz > n) continue;
    P::add1(a, P::weight(st, cb + k), P::load(xm + r3_slot(n, qx, qy, qz)));
  }
  typename P::T r = P::finish1(a);
  if constexpr (P::kPoison) {  // an input outside the float-float range: native fp64 row
    if (P::bad1(a)) r = native_row3d(xm, n, px, yy, z, st.d + cb);
  }
  y[cell * S + r3_slot(n, px, yy, z)] = r;
}

template <class P>
cudaError_t launch(const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s) {
  if (L.n_r3_tiles == 0) return cudaSuccess;
  const int64_t n_warps = (int64_t)L.n_r3_tiles * n_cells;
  const int64_t blocks = (n_warps * 32 + R3THREADS - 1) / R3THREADS;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  k_row3d<P><<<(unsigned)blocks, R3THREADS, 0, s>>>((const typename P::T*)x, (typename P::T*)y, L.r3_tiles,
                                                     L.n_r3_tiles, n_warps, L.slots_per_macro, L.n, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_rows = (L.n + 1) * (L.n + 2) / 2;
  k_row3d_lines<P><<<dim3((unsigned)((2 * n_rows + 127) / 128), (unsigned)n_cells), 128, 0, s>>>(
      (const typename P::T*)x, (typename P::T*)y, L.slots_per_macro, L.n, n_rows, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_row3d(int dtype, const LevelDev& L, int64_t n_cells, const void* x, void* y, cudaStream_t s) {
  switch (dtype) {
    case 1: return launch<ArF64FF>(L, n_cells, x, y, s);
    case 2: return launch<ArF32>(L, n_cells, x, y, s);
    case 3: return launch<ArF64Native>(L, n_cells, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
