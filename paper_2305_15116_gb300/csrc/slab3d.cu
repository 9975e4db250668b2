// 3D apply, shared-memory slab kernel: every point of a refined macro-tet
// (levels with n = 2^L <= 64).
//
// A macro array stacks triangular slices along z (slice z has side M = n+1-z
// and starts at T3(n+1) - T3(n+1-z), T3(k) = k(k+1)(k+2)/6); every slice is
// one contiguous range.  The 15-point stencil of the Kuhn refinement couples
// slice z only to slices z-1 and z+1 (offsets 0, ±(1,0,0), ±(0,1,0),
// ±(0,0,1), ±(1,-1,0), ±(1,0,-1), ±(0,1,-1), ±(1,-1,1)), so one CTA walks up a
// range of slices of one macro with three slices resident in shared memory —
// the paper's layer condition (Sec. 1.3, Sec. 5.2) one dimension up.  A fourth
// ring buffer receives the next slice by cp.async while the current one is
// computed (through a staging buffer and one split into float-float for the
// fp64 path), so each slice costs one barrier.
//
// For every slice the CTA writes ALL its points:
//  * interior points (x, y, z >= 1, x+y+z <= n-1): the full stencil of the
//    macro, weights in registers;
//  * points on the macro's own faces/edges/vertices: the macro's PARTIAL row
//    (the class stencil of the micro-elements inside this macro).  The
//    interface kernel then sums the copies' partials over the incident
//    macros (Sec. 5.1's interface primitives).
// Neighbour positions inside slice z (side M), slice z+1 (side M-1) and slice
// z-1 (side M+1) for point p = s(y) + x, s(y) = yM - y(y-1)/2:
//   z  : p±1, p+M-y (0,1,0), p+M-y-1 (-1,1,0), p-M+y-1 (0,-1,0), p-M+y (1,-1,0)
//   z+1: p-y (0,0,1), p-y-1 (-1,0,1), p-M (0,-1,1), p-M+1 (1,-1,1)
//   z-1: p+y (0,0,-1), p+y+1 (1,0,-1), p+M+1 (0,1,-1), p+M (-1,1,-1)
#include <mutex>

#include "arith.cuh"
#include "fallback.cuh"
#include "group.cuh"
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
// `direct`: the staged element is the memory element itself, so cp.async can
// land it in the ring without a conversion pass.
template <class P>
struct Stage;
template <>
struct Stage<ArF32> {
  using S = float;
  static constexpr bool direct = true;
  static __device__ __forceinline__ S from(float v) { return v; }
  static __device__ __forceinline__ float get(S s) { return s; }
  static __device__ __forceinline__ S zero() { return 0.0f; }
};
template <>
struct Stage<ArF64Native> {
  using S = double;
  static constexpr bool direct = true;
  static __device__ __forceinline__ S from(double v) { return v; }
  static __device__ __forceinline__ double get(S s) { return s; }
  static __device__ __forceinline__ S zero() { return 0.0; }
};
template <>
struct Stage<ArF64FF> {
  using S = float2;
  static constexpr bool direct = false;
  static __device__ __forceinline__ S from(double v) {
    const FF f = ff_split(v);
    return make_float2(f.h, f.l);
  }
  static __device__ __forceinline__ FF get(S s) { return FF{s.x, s.y}; }
  static __device__ __forceinline__ S zero() { return make_float2(0.0f, 0.0f); }
};

// Class weights as kept in shared memory, and the policy's weight type built
// from them (float-float: the two parts only; the packed forms are rebuilt in
// registers).
template <class P>
struct WStore;
template <>
struct WStore<ArF32> {
  using S = float;
  static __device__ __forceinline__ S load(const StencilPtr& st, int64_t i) { return __ldg(st.f + i); }
  static __device__ __forceinline__ ArF32::W w(S s) { return s; }
};
template <>
struct WStore<ArF64Native> {
  using S = double;
  static __device__ __forceinline__ S load(const StencilPtr& st, int64_t i) { return __ldg(st.d + i); }
  static __device__ __forceinline__ ArF64Native::W w(S s) { return s; }
};
template <>
struct WStore<ArF64FF> {
  using S = float2;
  static __device__ __forceinline__ S load(const StencilPtr& st, int64_t i) {
    return make_float2(__ldg(st.hi + i), __ldg(st.lo + i));
  }
  static __device__ __forceinline__ ArF64FF::W w(S s) {
    return ArF64FF::W{f2_pack(s.x, s.x), f2_pack(s.y, s.y), s.x, s.y};
  }
};

// Blocks per SM each kernel is built for (its register budget): 8-byte ring
// elements as shared memory allows at n = 64 (the float-float weights are kept
// as two floats and the next slice is staged in place, so that three blocks
// fit); fp32 without a bound (0: the compiler's own choice, 40 registers).
template <class P>
struct SlabOcc {
  static constexpr int value = 3;
};
template <>
struct SlabOcc<ArF32> {
  static constexpr int value = 0;
};

__device__ __forceinline__ int t3i(int k) { return k * (k + 1) * (k + 2) / 6; }
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

constexpr int NRING = 4;  // slices z-1, z, z+1 being read, z+2 being filled

// The work of one CTA: work item `it` = (macro, z0, z1) of a mesh whose
// vectors are x and y.
template <class P>
__device__ __forceinline__ void slab3d_item(const typename P::T* __restrict__ x, typename P::T* __restrict__ y,
                                            const int4 it, int n, int64_t S, int buf_elems, int guard,
                                            const StencilPtr st) {
  using SS = Stage<P>;
  using SV = typename SS::S;
  using T = typename P::T;
  using W = typename P::W;
  using WS = WStore<P>;
  using WSV = typename WS::S;
  // layout: [class weights: NCLS3*NW3 WSV] [ring: NRING x (guard + buf + guard) SV]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WSV* wcls = reinterpret_cast<WSV*>(smem_raw);
  SV* ring = reinterpret_cast<SV*>(smem_raw + (NCLS3 * NW3 * sizeof(WSV) + 15) / 16 * 16);
  const int stride = buf_elems + 2 * guard;
  // a slice staged raw (float-float) lands in its own ring buffer as T and
  // is converted in place by the thread that staged each element
  static_assert(SS::direct || sizeof(SV) == sizeof(T), "in-place staging needs equal element sizes");
  // offset of element 0 of slice z's buffer inside `ring`
  auto roff = [&](int z) -> int { return (z & (NRING - 1)) * stride + guard; };

  const int m = it.x, z0 = it.y, z1 = it.z;
  const T* __restrict__ xm = x + (int64_t)m * S;
  T* __restrict__ ym = y + (int64_t)m * S;
  const int N = n + 1;
  const int tid = threadIdx.x;

  // zero the ring (guards and stale tails must hold finite values), class weights
  for (int i = tid; i < NRING * stride; i += SLAB_THREADS) ring[i] = SS::zero();
  for (int i = tid; i < NCLS3 * NW3; i += SLAB_THREADS) wcls[i] = WS::load(st, (int64_t)m * (NCLS3 * NW3) + i);
  pdl_wait();  // x and y after the previous kernel in the stream (group.cuh)
  __syncthreads();
  // slices z0-1 .. z0+1 directly
  for (int z = max(z0 - 1, 0); z <= min(z0 + 1, n); ++z) {
    const int cnt = slice_count(n, z);
    const int off = t3i(N) - t3i(N - z);
    const int rb = roff(z);
    for (int i = tid; i < cnt; i += SLAB_THREADS) ring[rb + i] = SS::from(__ldg(xm + off + i));
  }
  // stage slice z0+2 (read when computing z0+1)
  auto stage = [&](int zs) {
    if (zs < z1 + 1 && zs <= n) {
      const int cnt = slice_count(n, zs);
      const int off = t3i(N) - t3i(N - zs);
      if (SS::direct) {
        const int rb = roff(zs);
        for (int i = tid; i < cnt; i += SLAB_THREADS) cp_async(&ring[rb + i], xm + off + i, sizeof(T));
      } else {
        T* raw = reinterpret_cast<T*>(ring + roff(zs));
        for (int i = tid; i < cnt; i += SLAB_THREADS) cp_async(raw + i, xm + off + i, sizeof(T));
      }
    }
    cp_async_commit();
  };
  stage(z0 + 2);
  __syncthreads();

  W w[NW3];  // interior weights (class 0) in registers
#pragma unroll
  for (int k = 0; k < NW3; ++k) w[k] = WS::w(wcls[k]);

  for (int z = z0; z < z1; ++z) {
    const int M = N - z;
    const int zoff = t3i(N) - t3i(N - z);
    const int bz = roff(z), bu = roff(z + 1), bd = roff(z - 1);

    // ---- the slice's work: interior units, then macro-boundary points -----
    // Interior points (x, y >= 1, x + y <= K = M - 2, z >= 1) come in units of
    // two adjacent points (x, y), (x + 1, y) of one row, x odd.  Rows are taken
    // in pairs (y, y + 1), y = 1 + 2r, which together hold K - 1 - 2r units;
    // r(K - r) units precede pair r, K/2 (K - K/2) in all.  The second point
    // of a unit at the end of an odd row lies on the macro's diagonal face: it
    // is evaluated (its neighbours are valid ring cells) but not written.
    // Macro-boundary points (z = 0: the whole slice, the face z = 0;
    // otherwise the rows y = 0, the column x = 0 and the diagonal x + y =
    // M - 1) get their partial rows; invalid neighbours carry weight 0 and
    // read guard cells or stale (finite) values.  Units and boundary points
    // cost about the same (a packed pair against one scalar float-float row)
    // and share one list, so that the threads reach the slice's barrier
    // together.
    {
      const int K = M - 2;
      const int units = (z >= 1 && M >= 4) ? (K / 2) * (K - K / 2) : 0;
      const int nb = (z == 0) ? M * (M + 1) / 2 : (M >= 2 ? 3 * (M - 1) : 1);
      const float Kf = (float)K;
      for (int wi = tid; wi < units + nb; wi += SLAB_THREADS) {
        if (wi < units) {
          const int u = wi;
          // row pair r: the largest r with r (K - r) <= u
          const float d = fmaxf(Kf * Kf - 4.0f * (float)u, 1.0f);
          int r = max((int)((Kf - d * rsqrtf(d)) * 0.5f), 0);
          if (r * (K - r) > u) --r;
          if ((r + 1) * (K - r - 1) <= u) ++r;
          const int j = u - r * (K - r);
          const int h = (K - 2 * r) >> 1;  // units in row 1 + 2r: ceil((K - 1 - 2r) / 2)
          const int yy = j < h ? 1 + 2 * r : 2 + 2 * r;
          const int xx = 1 + 2 * (j < h ? j : j - h);
          const int p = yy * M - (yy * (yy - 1)) / 2 + xx;
          // ring offsets of the first point in slices z, z+1, z-1; row gap A = M - y
          const int qz = bz + p, qu = bu + p - yy, qd = bd + p + yy, A = M - yy;
          auto at = [&](int i) { return P::pair(SS::get(ring[i]), SS::get(ring[i + 1])); };
          typename P::Acc a;
          P::first(a, w[0], at(qz));
          P::add_sym(a, w[1], at(qz + 1), at(qz - 1));           // (±1,0,0)
          P::add_sym(a, w[3], at(qz + A), at(qz - A - 1));       // (0,±1,0)
          P::add_sym(a, w[5], at(qz - A), at(qz + A - 1));       // ±(1,-1,0)
          P::add_sym(a, w[7], at(qu), at(qd));                   // (0,0,±1)
          P::add_sym(a, w[8], at(qu - 1), at(qd + 1));           // ±(-1,0,1)
          P::add_sym(a, w[9], at(qu - A), at(qd + A + 1));       // ±(0,-1,1)
          P::add_sym(a, w[10], at(qu - A + 1), at(qd + A));      // ±(1,-1,1)
          T r0, r1;
          P::finish(a, r0, r1);
          if constexpr (P::kPoison) {
            if (P::bad(a)) {  // an input outside the float-float range: native fp64 rows
              const double* wd = st.d + (int64_t)m * (NCLS3 * NW3);
              r0 = native_row3d(xm, n, xx, yy, z, wd);
              if (xx < K - yy) r1 = native_row3d(xm, n, xx + 1, yy, z, wd);
            }
          }
          ym[zoff + p] = r0;
          if (xx < K - yy) ym[zoff + p + 1] = r1;
        } else {
          const int q = wi - units;
          int xx, yv;
          if (z == 0) {
            yv = tri_row(q, M);
            xx = q - (yv * M - (yv * (yv - 1)) / 2);
          } else if (M == 1) {
            xx = 0;
            yv = 0;
          } else if (q < M) {  // y = 0
            xx = q;
            yv = 0;
          } else if (q < 2 * M - 1) {  // x = 0, y = 1 .. M-1
            xx = 0;
            yv = q - M + 1;
          } else {  // diagonal, y = 1 .. M-2
            yv = q - (2 * M - 1) + 1;
            xx = M - 1 - yv;
          }
          const int cls = (xx == 0 ? 1 : 0) | (yv == 0 ? 2 : 0) | (z == 0 ? 4 : 0) | (xx + yv == M - 1 ? 8 : 0);
          const int p = yv * M - (yv * (yv - 1)) / 2 + xx;
          const WSV* cwv = wcls + cls * NW3;
          auto cw = [&](int k) { return WS::w(cwv[k]); };
          const int qz = bz + p, qu = bu + p - yv, qd = bd + p + yv, A = M - yv;
          typename P::Acc1 a;
          P::first1(a, cw(0), SS::get(ring[qz]));
          P::add1(a, cw(1), SS::get(ring[qz + 1]));
          P::add1(a, cw(2), SS::get(ring[qz - 1]));
          P::add1(a, cw(3), SS::get(ring[qz + A]));
          P::add1(a, cw(4), SS::get(ring[qz - A - 1]));
          P::add1(a, cw(5), SS::get(ring[qz - A]));
          P::add1(a, cw(6), SS::get(ring[qz + A - 1]));
          P::add1(a, cw(7), SS::get(ring[qu]));
          P::add1(a, cw(8), SS::get(ring[qu - 1]));
          P::add1(a, cw(9), SS::get(ring[qu - A]));
          P::add1(a, cw(10), SS::get(ring[qu - A + 1]));
          P::add1(a, cw(11), SS::get(ring[qd]));
          P::add1(a, cw(12), SS::get(ring[qd + 1]));
          P::add1(a, cw(13), SS::get(ring[qd + A + 1]));
          P::add1(a, cw(14), SS::get(ring[qd + A]));
          T r = P::finish1(a);
          if constexpr (P::kPoison) {
            if (P::bad1(a)) r = native_row3d(xm, n, xx, yv, z, st.d + ((int64_t)m * NCLS3 + cls) * NW3);
          }
          ym[zoff + p] = r;
        }
      }
    }
    // slice z+2 has landed (staged during the previous iteration): convert it
    // into its ring buffer when it was staged raw; then one barrier publishes
    // it and retires slice z-1, whose buffer receives slice z+3.
    cp_async_wait_all();
    if (!SS::direct && z + 2 < z1 + 1 && z + 2 <= n) {
      const int cnt = slice_count(n, z + 2);
      const int rb = roff(z + 2);
      const T* raw = reinterpret_cast<const T*>(ring + rb);
      for (int i = tid; i < cnt; i += SLAB_THREADS) ring[rb + i] = SS::from(raw[i]);
    }
    __syncthreads();
    stage(z + 3);
  }
  cp_async_wait_all();
}

template <class P>
__global__ void __launch_bounds__(SLAB_THREADS, SlabOcc<P>::value) k_slab3d(const typename P::T* __restrict__ x,
                                                         typename P::T* __restrict__ y,
                                                         const int4* __restrict__ items, int n, int64_t S,
                                                         int buf_elems, int guard, StencilPtr st) {
  pdl_trigger();
  slab3d_item<P>(x, y, items[blockIdx.x], n, S, buf_elems, guard, st);
}

// Several meshes in one launch: each owns a consecutive range of the blocks
// (one per work item, as in its own launch) and a block finds its mesh by
// binary search over the ranges.  The meshes share n (the shared-memory
// layout).
struct SlabDesc {
  const void* x;
  void* y;
  const int4* items;
  int64_t S;
  StencilPtr st;
  int block_begin;
};
struct SlabGroup {
  SlabDesc d[kGroupMax];
  int count, n, buf_elems, guard;
};

template <class P>
__global__ void __launch_bounds__(SLAB_THREADS, SlabOcc<P>::value) k_slab3d_group(const __grid_constant__ SlabGroup g) {
  pdl_trigger();
  int lo = 0, hi = g.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.d[mid].block_begin <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  const SlabDesc& d = g.d[lo];
  slab3d_item<P>(static_cast<const typename P::T*>(d.x), static_cast<typename P::T*>(d.y),
                 d.items[(int)blockIdx.x - d.block_begin], g.n, d.S, g.buf_elems, g.guard, d.st);
}

// The shared-memory limit is a property of the kernel shared by every thread
// and stream of the process: raise it once, to what the largest slab level
// (n = 64) needs, so that concurrent launches for different levels never see
// a limit set for another level.
template <class P>
cudaError_t ensure_attr() {
  using SV = typename Stage<P>::S;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    constexpr int nmax = 64;
    const int bmax = (nmax + 1) * (nmax + 2) / 2;
    const size_t wb = ((size_t)NCLS3 * NW3 * sizeof(typename WStore<P>::S) + 15) / 16 * 16;
    const size_t rb = ((size_t)NRING * (bmax + 2 * (nmax + 3)) * sizeof(SV) + 15) / 16 * 16;
    attr = cudaFuncSetAttribute(k_slab3d<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(wb + rb));
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_slab3d_group<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(wb + rb));
  });
  return attr;
}

template <class P>
cudaError_t launch_items(const LevelDev& L, const int4* items, int n_items, const void* x, void* y, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  using SV = typename Stage<P>::S;
  const int n = L.n;
  const int buf = (n + 1) * (n + 2) / 2;
  const int guard = n + 3;
  const size_t w_bytes = ((size_t)NCLS3 * NW3 * sizeof(typename WStore<P>::S) + 15) / 16 * 16;
  const size_t ring_bytes = ((size_t)NRING * (buf + 2 * guard) * sizeof(SV) + 15) / 16 * 16;
  const size_t bytes = w_bytes + ring_bytes;
  const cudaError_t attr = ensure_attr<P>();
  if (attr != cudaSuccess) return attr;
  if (n > 64) return cudaErrorInvalidValue;
  StencilPtr st{L.st64, L.st32, L.st_hi, L.st_lo};
  return launch_pdl(k_slab3d<P>, dim3(n_items), dim3(SLAB_THREADS), bytes, s, (const typename P::T*)x,
                    (typename P::T*)y, items, n, L.slots_per_macro, buf, guard, st);
}

template <class P>
cudaError_t launch_group_t(const Mesh* const* ms, const int* levels, const void* const* xs, void* const* ys,
                           int count, int dt, cudaStream_t s) {
  using SV = typename Stage<P>::S;
  const int n = ms[0]->levels[levels[0]].n;
  if (n > 64) return cudaErrorInvalidValue;
  const int buf = (n + 1) * (n + 2) / 2;
  const int guard = n + 3;
  const size_t w_bytes = ((size_t)NCLS3 * NW3 * sizeof(typename WStore<P>::S) + 15) / 16 * 16;
  const size_t ring_bytes = ((size_t)NRING * (buf + 2 * guard) * sizeof(SV) + 15) / 16 * 16;
  const cudaError_t attr = ensure_attr<P>();
  if (attr != cudaSuccess) return attr;
  SlabGroup g;
  g.n = n;
  g.buf_elems = buf;
  g.guard = guard;
  for (int i0 = 0; i0 < count;) {
    g.count = 0;
    int blocks = 0;
    int i = i0;
    for (; i < count && g.count < kGroupMax; ++i) {
      const LevelDev& L = ms[i]->levels[levels[i]];
      if (L.n != n || L.n_slabs == 0) return cudaErrorInvalidValue;
      const bool tuned = L.slabs_dt[dt] != nullptr;
      const int n_items = tuned ? L.n_slabs_dt[dt] : L.n_slabs;
      SlabDesc& d = g.d[g.count++];
      d.x = xs[i];
      d.y = ys[i];
      d.items = tuned ? L.slabs_dt[dt] : L.slabs;
      d.S = L.slots_per_macro;
      d.st = StencilPtr{L.st64, L.st32, L.st_hi, L.st_lo};
      d.block_begin = blocks;
      blocks += n_items;
    }
    i0 = i;
    const cudaError_t e = launch_pdl(k_slab3d_group<P>, dim3(blocks), dim3(SLAB_THREADS), w_bytes + ring_bytes, s, g);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// the level's work list for element type dt (the autotuned one when present)
template <class P>
cudaError_t launch_t(const LevelDev& L, int dt, const void* x, void* y, cudaStream_t s) {
  if (L.n_slabs == 0) return cudaSuccess;
  return L.slabs_dt[dt] ? launch_items<P>(L, L.slabs_dt[dt], L.n_slabs_dt[dt], x, y, s)
                        : launch_items<P>(L, L.slabs, L.n_slabs, x, y, s);
}

}  // namespace

cudaError_t slab3d_prepare() {
  cudaError_t e = ensure_attr<ArF64FF>();
  if (e == cudaSuccess) e = ensure_attr<ArF32>();
  if (e == cudaSuccess) e = ensure_attr<ArF64Native>();
  return e;
}

cudaError_t launch_slab3d_items(int dtype, const LevelDev& L, const int4* items, int n_items, const void* x,
                                void* y, cudaStream_t s) {
  switch (dtype) {
    case 1: return launch_items<ArF64FF>(L, items, n_items, x, y, s);
    case 2: return launch_items<ArF32>(L, items, n_items, x, y, s);
    case 3: return launch_items<ArF64Native>(L, items, n_items, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_slab3d_group(int dtype, const Mesh* const* ms, const int* levels, const void* const* xs,
                                void* const* ys, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  switch (dtype) {
    case 1: return launch_group_t<ArF64FF>(ms, levels, xs, ys, count, 1, s);
    case 2: return launch_group_t<ArF32>(ms, levels, xs, ys, count, 2, s);
    case 3: return launch_group_t<ArF64Native>(ms, levels, xs, ys, count, 3, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_slab3d(int dtype, const LevelDev& L, const void* x, void* y, cudaStream_t s) {
  switch (dtype) {
    case 1: return launch_t<ArF64FF>(L, 1, x, y, s);
    case 2: return launch_t<ArF32>(L, 2, x, y, s);
    case 3: return launch_t<ArF64Native>(L, 3, x, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hyteg
