// 3D apply, shared-memory slab kernel: every point of a refined macro-tet
// (levels with n = 2^L <= 64).
//
// A macro array stacks triangular slices along z (slice z has side M = n+1-z
// and starts at T3(n+1) - T3(n+1-z), T3(k) = k(k+1)(k+2)/6); every slice is
// one contiguous range.  The 15-point stencil of the Kuhn refinement couples
// slice z only to slices z-1 and z+1 (offsets 0, ±(1,0,0), ±(0,1,0),
// ±(0,0,1), ±(1,-1,0), ±(1,0,-1), ±(0,1,-1), ±(1,-1,1)), so one CTA walks up a
// range of slices of one macro with three slices resident in shared memory —
// the paper's layer condition (Sec. 2.3, Sec. 4.2) one dimension up.  The next
// slice is staged with cp.async while the current one is computed, then split
// once (float-float path) into the ring.
//
// For every slice the CTA writes ALL its points:
//  * interior points (x, y, z >= 1, x+y+z <= n-1): the full stencil of the
//    macro, weights in registers;
//  * points on the macro's own faces/edges/vertices: the macro's PARTIAL row
//    (the class stencil of the micro-elements inside this macro).  The
//    interface kernel then sums the copies' partials over the incident
//    macros (Sec. 4.1's interface primitives).
// Neighbour positions inside slice z (side M), slice z+1 (side M-1) and slice
// z-1 (side M+1) for point p = s(y) + x, s(y) = yM - y(y-1)/2:
//   z  : p±1, p+M-y (0,1,0), p+M-y-1 (-1,1,0), p-M+y-1 (0,-1,0), p-M+y (1,-1,0)
//   z+1: p-y (0,0,1), p-y-1 (-1,0,1), p-M (0,-1,1), p-M+1 (1,-1,1)
//   z-1: p+y (0,0,-1), p+y+1 (1,0,-1), p+M+1 (0,1,-1), p+M (-1,1,-1)
#include "arith.cuh"
#include "hyteg_internal.h"

namespace hyteg {

namespace {

constexpr int SLAB_THREADS = 256;

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory element of a staged point and its conversion from memory.
template <class P>
struct Stage;
template <>
struct Stage<ArF32> {
  using S = float;
  static __device__ __forceinline__ S from(float v) { return v; }
  static __device__ __forceinline__ float get(S s) { return s; }
  static __device__ __forceinline__ S zero() { return 0.0f; }
};
template <>
struct Stage<ArF64Native> {
  using S = double;
  static __device__ __forceinline__ S from(double v) { return v; }
  static __device__ __forceinline__ double get(S s) { return s; }
  static __device__ __forceinline__ S zero() { return 0.0; }
};
template <>
struct Stage<ArF64FF> {
  using S = float2;
  static __device__ __forceinline__ S from(double v) {
    const FF f = ff_split(v);
    return make_float2(f.h, f.l);
  }
  static __device__ __forceinline__ FF get(S s) { return FF{s.x, s.y}; }
  static __device__ __forceinline__ S zero() { return make_float2(0.0f, 0.0f); }
};

__device__ __forceinline__ int64_t t3(int64_t k) { return k * (k + 1) * (k + 2) / 6; }
__device__ __forceinline__ int slice_count(int n, int z) {
  const int M = n + 1 - z;
  return M * (M + 1) / 2;
}

// Row y of the points q = 0.. of a triangle whose row j (j = 0..) holds K - j
// points: the largest y with y K - y(y-1)/2 <= q.
__device__ __forceinline__ int tri_row(int q, int K) {
  const float b = 2.0f * K + 1.0f;
  int y = (int)((b - sqrtf(b * b - 8.0f * q)) * 0.5f);
  y = max(y, 0);
  if (y * K - (y * (y - 1)) / 2 > q) --y;
  if ((y + 1) * K - ((y + 1) * y) / 2 <= q) ++y;
  return y;
}

template <class P>
__global__ void __launch_bounds__(SLAB_THREADS) k_slab3d(const typename P::T* __restrict__ x,
                                                         typename P::T* __restrict__ y,
                                                         const int4* __restrict__ items, int n, int64_t S,
                                                         int buf_elems, int guard, StencilPtr st) {
  using SS = Stage<P>;
  using SV = typename SS::S;
  using T = typename P::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: [raw staging: buf_elems T] [3 ring buffers: (guard + buf_elems + guard) SV]
  T* raw = reinterpret_cast<T*>(smem_raw);
  SV* ring0 = reinterpret_cast<SV*>(smem_raw + ((size_t)buf_elems * sizeof(T) + 15) / 16 * 16);
  const int stride = buf_elems + 2 * guard;
  auto ring = [&](int z) -> SV* { return ring0 + (size_t)(((z % 3) + 3) % 3) * stride + guard; };
  // class stencils of this macro (16 classes x 15 weights)
  typename P::W* wcls = reinterpret_cast<typename P::W*>(
      reinterpret_cast<unsigned char*>(ring0) + ((3 * (size_t)stride * sizeof(SV) + 15) / 16 * 16));

  const int4 it = items[blockIdx.x];
  const int m = it.x, z0 = it.y, z1 = it.z;
  const T* __restrict__ xm = x + (int64_t)m * S;
  T* __restrict__ ym = y + (int64_t)m * S;
  const int N = n + 1;
  const int tid = threadIdx.x;

  // zero the ring (guards and stale tails must hold finite values)
  for (int i = tid; i < 3 * stride; i += SLAB_THREADS) ring0[i] = SS::zero();
  for (int i = tid; i < NCLS3 * NW3; i += SLAB_THREADS) wcls[i] = P::weight(st, (int64_t)m * (NCLS3 * NW3) + i);
  __syncthreads();
  // load slices z0-1 .. z0+1 synchronously
  for (int z = max(z0 - 1, 0); z <= min(z0 + 1, n); ++z) {
    const int cnt = slice_count(n, z);
    const int64_t off = t3(N) - t3(N - z);
    SV* b = ring(z);
    for (int i = tid; i < cnt; i += SLAB_THREADS) b[i] = SS::from(__ldg(xm + off + i));
  }
  __syncthreads();

  // interior weights (class 0) in registers
  const int64_t wb = (int64_t)m * (NCLS3 * NW3);
  typename P::W w[NW3];
#pragma unroll
  for (int k = 0; k < NW3; ++k) w[k] = P::weight(st, wb + k);
  const int warp = tid >> 5, lane = tid & 31;

  for (int z = z0; z < z1; ++z) {
    // stage slice z+2 asynchronously (needed when computing slice z+1)
    const bool pre = (z + 1 < z1) && (z + 2 <= n);
    if (pre) {
      const int cnt = slice_count(n, z + 2);
      const int64_t off = t3(N) - t3(N - z - 2);
      for (int i = tid; i < cnt; i += SLAB_THREADS) cp_async(raw + i, xm + off + i, sizeof(T));
      cp_async_commit();
    }
    const int M = N - z;
    const int64_t zoff = t3(N) - t3(N - z);
    const SV* __restrict__ bz = ring(z);
    const SV* __restrict__ bu = ring(z + 1);
    const SV* __restrict__ bd = ring(z - 1);

    // ---- interior points: x, y >= 1, x + y <= K = M - 2 (z >= 1) ---------
    // Row y holds K - y points; rows y and K - y together hold K <= 63
    // points, so one warp takes such a pair and each lane two points
    // (positions lane and lane + 32), evaluated together.
    if (z >= 1 && M >= 4) {
      const int K = M - 2;
      const int units = K / 2;  // pairs y = 1 .. (K-1)/2, plus the middle row when K is even
      for (int u = warp; u < units; u += SLAB_THREADS / 32) {
        const int ya = u + 1, yb = K - ya;  // yb == ya: the middle row, alone
        const int la = K - ya;              // points in row ya
        const int total = (ya == yb) ? la : K;
        int px[2], py[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int t = min(lane + 32 * h, total - 1);  // out-of-range lanes repeat a valid point
          const bool first_row = t < la;
          py[h] = first_row ? ya : yb;
          px[h] = first_row ? t + 1 : t - la + 1;
        }
        int p[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) p[h] = py[h] * M - (py[h] * (py[h] - 1)) / 2 + px[h];
        auto at = [&](const SV* b, int i0, int i1) { return P::pair(SS::get(b[i0]), SS::get(b[i1])); };
        typename P::Acc a;
        P::first(a, w[0], at(bz, p[0], p[1]));
        P::add_sym(a, w[1], at(bz, p[0] + 1, p[1] + 1), at(bz, p[0] - 1, p[1] - 1));
        P::add_sym(a, w[3], at(bz, p[0] + M - py[0], p[1] + M - py[1]),
                   at(bz, p[0] - M + py[0] - 1, p[1] - M + py[1] - 1));
        P::add_sym(a, w[5], at(bz, p[0] - M + py[0], p[1] - M + py[1]),
                   at(bz, p[0] + M - py[0] - 1, p[1] + M - py[1] - 1));
        P::add_sym(a, w[7], at(bu, p[0] - py[0], p[1] - py[1]), at(bd, p[0] + py[0], p[1] + py[1]));
        P::add_sym(a, w[8], at(bu, p[0] - py[0] - 1, p[1] - py[1] - 1), at(bd, p[0] + py[0] + 1, p[1] + py[1] + 1));
        P::add_sym(a, w[9], at(bu, p[0] - M, p[1] - M), at(bd, p[0] + M + 1, p[1] + M + 1));
        P::add_sym(a, w[10], at(bu, p[0] - M + 1, p[1] - M + 1), at(bd, p[0] + M, p[1] + M));
        T r0, r1;
        P::finish(a, r0, r1);
        if (lane < total) ym[zoff + p[0]] = r0;
        if (lane + 32 < total) ym[zoff + p[1]] = r1;
      }
    }
    // ---- macro-boundary points of the slice: partial rows ---------------------
    // z = 0: the whole slice lies on the face z = 0; otherwise the rows y = 0,
    // the column x = 0 and the diagonal x + y = M - 1.
    {
      const int nb = (z == 0) ? M * (M + 1) / 2 : (M >= 2 ? 3 * (M - 1) : 1);
      for (int q = tid; q < nb; q += SLAB_THREADS) {
        int xx, yy;
        if (z == 0) {
          yy = tri_row(q, M);
          xx = q - (yy * M - (yy * (yy - 1)) / 2);
        } else if (M == 1) {
          xx = 0;
          yy = 0;
        } else if (q < M) {  // y = 0
          xx = q;
          yy = 0;
        } else if (q < 2 * M - 1) {  // x = 0, y = 1 .. M-1
          xx = 0;
          yy = q - M + 1;
        } else {  // diagonal, y = 1 .. M-2
          yy = q - (2 * M - 1) + 1;
          xx = M - 1 - yy;
        }
        const int cls = (xx == 0 ? 1 : 0) | (yy == 0 ? 2 : 0) | (z == 0 ? 4 : 0) | (xx + yy == M - 1 ? 8 : 0);
        const int p = yy * M - (yy * (yy - 1)) / 2 + xx;
        const typename P::W* cw = wcls + cls * NW3;
        // invalid neighbours carry weight 0 and read guard or stale (finite) values
        typename P::Acc1 a;
        P::first1(a, cw[0], SS::get(bz[p]));
        P::add1(a, cw[1], SS::get(bz[p + 1]));
        P::add1(a, cw[2], SS::get(bz[p - 1]));
        P::add1(a, cw[3], SS::get(bz[p + M - yy]));
        P::add1(a, cw[4], SS::get(bz[p - M + yy - 1]));
        P::add1(a, cw[5], SS::get(bz[p - M + yy]));
        P::add1(a, cw[6], SS::get(bz[p + M - yy - 1]));
        P::add1(a, cw[7], SS::get(bu[p - yy]));
        P::add1(a, cw[8], SS::get(bu[p - yy - 1]));
        P::add1(a, cw[9], SS::get(bu[p - M]));
        P::add1(a, cw[10], SS::get(bu[p - M + 1]));
        P::add1(a, cw[11], SS::get(bd[p + yy]));
        P::add1(a, cw[12], SS::get(bd[p + yy + 1]));
        P::add1(a, cw[13], SS::get(bd[p + M + 1]));
        P::add1(a, cw[14], SS::get(bd[p + M]));
        ym[zoff + p] = P::finish1(a);
      }
    }
    if (pre) cp_async_wait_all();
    __syncthreads();  // slice z-1 is no longer read; staged slice z+2 has landed
    if (pre) {
      const int cnt = slice_count(n, z + 2);
      SV* b = ring(z + 2);
      for (int i = tid; i < cnt; i += SLAB_THREADS) b[i] = SS::from(raw[i]);
    }
    __syncthreads();
  }
}

template <class P>
cudaError_t launch_t(const LevelDev& L, const void* x, void* y, cudaStream_t s) {
  if (L.n_slabs == 0) return cudaSuccess;
  using SV = typename Stage<P>::S;
  const int n = L.n;
  const int buf = (n + 1) * (n + 2) / 2;
  const int guard = n + 3;
  const size_t raw_bytes = ((size_t)buf * sizeof(typename P::T) + 15) / 16 * 16;
  const size_t ring_bytes = (3 * (size_t)(buf + 2 * guard) * sizeof(SV) + 15) / 16 * 16;
  const size_t bytes = raw_bytes + ring_bytes + (size_t)NCLS3 * NW3 * sizeof(typename P::W);
  cudaError_t e = cudaFuncSetAttribute(k_slab3d<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  k_slab3d<P><<<L.n_slabs, SLAB_THREADS, bytes, s>>>((const typename P::T*)x, (typename P::T*)y, L.slabs, n,
                                                    L.slots_per_macro, buf, guard, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_slab3d(int dtype, const LevelDev& L, const void* x, void* y, cudaStream_t s) {
  switch (dtype) {
    case 1: return launch_t<ArF64FF>(L, x, y, s);
    case 2: return launch_t<ArF32>(L, x, y, s);
    case 3: return launch_t<ArF64Native>(L, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
