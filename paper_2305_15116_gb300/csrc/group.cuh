// Launching one kernel over the vectors of several meshes (a group).
//
// A kernel body is written once, as Body::run(prm, block, n_blocks): the
// work of block `block` of the `n_blocks` blocks that one mesh's part of the
// launch has.  k_group<Body, N> runs it for up to N meshes: each mesh owns a
// consecutive range of the launch's blocks (its own block count, the same as
// when it is launched alone), a block finds its mesh by binary search over
// the ranges, and the parameters travel in the kernel's parameter block, so
// a launch allocates nothing.  A mesh launched alone uses N = 1 and the same
// body, so its arithmetic is that of the group launch.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

namespace hyteg {

// ---- programmatic dependent launch ------------------------------------------
// The solve's kernels are launched so that a kernel may start while the one
// before it in the stream finishes (Hopper/Blackwell programmatic stream
// serialisation): every kernel lets its dependents launch as soon as all its
// blocks have started (pdl_trigger), and reads only tables that no kernel
// writes (work lists, incidences, stencils) before pdl_wait, which returns
// once the previous kernel has completed and its writes are visible.  Every
// access to vectors comes after pdl_wait.  A kernel launched without the
// attribute, or after a non-kernel operation, finds pdl_wait satisfied.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// A body that reads tables before its vectors declares kLateWait = true and
// calls pdl_wait itself; every other body runs after pdl_wait.
template <class B, class = void>
struct late_wait : std::false_type {};
template <class B>
struct late_wait<B, std::void_t<decltype(B::kLateWait)>> : std::bool_constant<B::kLateWait> {};

constexpr int kGroupMax = 16;  // meshes per group launch

template <class Prm, int N>
struct GroupArgs {
  Prm p[N];
  int begin[N + 1];  // first block of every mesh; begin[count] = the launch's blocks
  int count;
};

template <class Prm, int N>
__device__ __forceinline__ int group_entry(const GroupArgs<Prm, N>& g, int block) {
  int lo = 0, hi = g.count - 1;  // the last mesh whose range starts at or before `block`
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.begin[mid] <= block)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <class Body, int N>
__global__ void __launch_bounds__(Body::kThreads) k_group(const __grid_constant__ GroupArgs<typename Body::Prm, N> g) {
  pdl_trigger();
  if constexpr (!late_wait<Body>::value) pdl_wait();
  const int e = N == 1 ? 0 : group_entry(g, (int)blockIdx.x);
  Body::run(g.p[e], (int)blockIdx.x - g.begin[e], g.begin[e + 1] - g.begin[e]);
}

// Launches Body over `count` meshes, blocks[i] blocks for mesh i (meshes with
// no blocks are skipped), in launches of at most kGroupMax meshes.
template <class Body>
cudaError_t launch_group(const typename Body::Prm* p, const int* blocks, int count, cudaStream_t s,
                         size_t smem = 0) {
  using Prm = typename Body::Prm;
  if (count == 1) {
    if (blocks[0] <= 0) return cudaSuccess;
    GroupArgs<Prm, 1> g;
    g.p[0] = p[0];
    g.begin[0] = 0;
    g.begin[1] = blocks[0];
    g.count = 1;
    return launch_pdl(k_group<Body, 1>, dim3((unsigned)blocks[0]), dim3(Body::kThreads), smem, s, g);
  }
  for (int i0 = 0; i0 < count;) {
    GroupArgs<Prm, kGroupMax> g;
    g.count = 0;
    long long total = 0;
    int i = i0;
    for (; i < count && g.count < kGroupMax; ++i) {
      if (blocks[i] <= 0) continue;
      if (total + blocks[i] > 0x7FFFFFFF) break;
      g.p[g.count] = p[i];
      g.begin[g.count] = (int)total;
      total += blocks[i];
      ++g.count;
    }
    if (i == i0) return cudaErrorInvalidValue;  // one mesh alone exceeds the grid limit
    i0 = i;
    if (g.count == 0) continue;
    g.begin[g.count] = (int)total;
    const cudaError_t e =
        launch_pdl(k_group<Body, kGroupMax>, dim3((unsigned)total), dim3(Body::kThreads), smem, s, g);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hyteg
