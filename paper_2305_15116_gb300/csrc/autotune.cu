// Autotuners run at refinement: the 3D slab kernel's work split (z-ranges
// per macro-tet) and the 2D kernel's tile height.
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "hyteg_internal.h"

namespace hyteg {

// ---- autotuner of the slab work split -------------------------------------------
// How many z-ranges a macro is cut into trades the waves of CTAs over the SMs
// (which depend on the blocks per SM of each element type) against the
// per-item cost of loading the first three slices.  On first use of a level
// size the kernel is timed for each candidate on scratch vectors (the best
// of two launches each, so that a concurrent workload inflates no candidate
// in particular) and the fastest list is kept; the choice is cached per
// (macro count, level, element type) for the process.  Float-float and fp32
// are timed; native fp64, which fits the same blocks per SM as float-float,
// takes float-float's choice.  Levels below 2^20 slots keep two z-ranges:
// their kernels take a few microseconds, and a solve server meets many such
// sizes once each.
cudaError_t slab3d_autotune(Mesh& m, LevelDev& L) {
  if (L.n_slabs == 0 || m.autotune == 0) return cudaSuccess;
  const int64_t total = L.slots_per_macro * m.n_cells;
  if (total < (int64_t(1) << 20)) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::array<int64_t, 3>, int> cache;
  constexpr int kCand[] = {2, 3, 4, 5, 6, 8};
  void* x = nullptr;
  void* y = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaSuccess;
  auto cleanup = [&] {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) {  // nothing of the timing may still run when the scratch is released
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    dev_free(m, x);
    dev_free(m, y);
  };
  for (int dt = 1; dt <= 3 && err == cudaSuccess; ++dt) {
    const std::array<int64_t, 3> key{m.n_cells, L.n, dt == 3 ? 1 : dt};
    int best = dt == 3 ? L.slab_chunks[1] : 0;
    if (best == 0) {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) best = it->second;
    }
    if (best == 0 && m.autotune < 2) continue;  // lookup only: the default split
    if (best == 0) {
      if (!x) {
        // no room for the scratch vectors: keep the default split
        void* p = nullptr;
        if (dev_alloc(m, &p, sizeof(double) * total) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        x = p;
        p = nullptr;
        if (dev_alloc(m, &p, sizeof(double) * total) != cudaSuccess) {
          cudaGetLastError();
          break;  // x is released below
        }
        y = p;
        if ((err = dev_zero(m, x, sizeof(double) * total)) != cudaSuccess) break;
        if ((err = dev_sync(m)) != cudaSuccess) break;
        if ((err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((err = cudaEventCreate(&e0)) != cudaSuccess) break;
        if ((err = cudaEventCreate(&e1)) != cudaSuccess) break;
      }
      float best_ms = 0.0f;
      for (int c : kCand) {
        const std::vector<int4> items = slab_work_list(L.n, m.n_cells, c);
        int4* d_items = nullptr;
        if ((err = dev_alloc(m, (void**)&d_items, items.size() * sizeof(int4))) != cudaSuccess) break;
        err = dev_upload(m, d_items, items.data(), items.size() * sizeof(int4));
        if (err == cudaSuccess) err = dev_sync(m);
        float ms = 0.0f;
        const int first = c == kCand[0] ? 0 : 1;  // one warm-up launch per element type
        for (int rep = first; rep < 3 && err == cudaSuccess; ++rep) {
          if ((err = cudaEventRecord(e0, s)) != cudaSuccess) break;
          if ((err = launch_slab3d_items(dt, L, d_items, int(items.size()), x, y, s)) != cudaSuccess) break;
          if ((err = cudaEventRecord(e1, s)) != cudaSuccess) break;
          if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
          float t = 0.0f;
          if ((err = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
          if (rep == 1 || (rep > 1 && t < ms)) ms = t;
        }
        const cudaError_t ef = cudaStreamSynchronize(s);
        dev_free(m, d_items);
        if (err == cudaSuccess) err = ef;
        if (err != cudaSuccess) break;
        if (best == 0 || ms < best_ms) {
          best = c;
          best_ms = ms;
        }
      }
      if (err != cudaSuccess) break;
      std::lock_guard<std::mutex> lk(mu);
      cache[key] = best;
    }
    if (best != 2) {  // the default list holds two z-ranges per macro
      const std::vector<int4> items = slab_work_list(L.n, m.n_cells, best);
      if ((err = dev_alloc(m, (void**)&L.slabs_dt[dt], items.size() * sizeof(int4))) != cudaSuccess) break;
      if ((err = dev_upload(m, L.slabs_dt[dt], items.data(), items.size() * sizeof(int4))) != cudaSuccess) break;
      L.n_slabs_dt[dt] = int(items.size());
    }
    L.slab_chunks[dt] = best;
  }
  if (err == cudaSuccess) err = dev_sync(m);
  cleanup();
  return err;
}

// ---- autotuner of the 2D tile shape ----------------------------------------------
// A warp walks the rows of its tile one after another (three rows in
// registers, the next ones in flight), so the rows per tile trade the
// number of serial walks and their balance over the SMs against the cost of
// starting a walk (its halo rows and the first rows in flight).  The best
// height differs per element type and level (measured at level 11 on 32
// macros: float-float flat from 16 to 64 rows, fp32 best at 16).  On first
// use of a level size of at least 2^20 slots the apply kernel is timed for
// 8, 16, 32 and 64 rows (best of two launches after a warm-up) on scratch
// vectors, per element type, and the fastest list is kept (cached per macro
// count, level and element type for the process).  Smaller levels keep the
// default lists (their kernels take microseconds, and the chunk already
// shrinks until the level has 16 tiles per SM).
cudaError_t tiles2d_autotune(Mesh& m, LevelDev& L) {
  if (m.dim != 2 || m.autotune == 0) return cudaSuccess;
  const int64_t total = L.slots_per_macro * m.n_cells;
  if (total < (int64_t(1) << 20) || L.n < 64) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::array<int64_t, 3>, int> cache;
  constexpr int kCand[] = {8, 16, 32, 64};
  void* x = nullptr;
  void* y = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaSuccess;
  auto cleanup = [&] {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) {  // nothing of the timing may still run when the scratch is released
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    dev_free(m, x);
    dev_free(m, y);
  };
  for (int dt = 1; dt <= 3 && err == cudaSuccess; ++dt) {
    const std::array<int64_t, 3> key{m.n_cells, L.n, dt};
    int best = 0;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) best = it->second;
    }
    if (best == 0 && m.autotune < 2) continue;  // lookup only: the default list
    if (best == 0) {
      if (!x) {
        // no room for the scratch vectors: keep the default lists
        void* p = nullptr;
        if (dev_alloc(m, &p, sizeof(double) * total) != cudaSuccess) {
          cudaGetLastError();
          break;
        }
        x = p;
        p = nullptr;
        if (dev_alloc(m, &p, sizeof(double) * total) != cudaSuccess) {
          cudaGetLastError();
          break;  // x is released below
        }
        y = p;
        if ((err = dev_zero(m, x, sizeof(double) * total)) != cudaSuccess) break;
        if ((err = dev_sync(m)) != cudaSuccess) break;
        if ((err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((err = cudaEventCreate(&e0)) != cudaSuccess) break;
        if ((err = cudaEventCreate(&e1)) != cudaSuccess) break;
      }
      float best_ms = 0.0f;
      for (int c : kCand) {
        const std::vector<int4> tl = tile_list_2d(L.n, c, kTileWidth2);
        int4* d_tiles = nullptr;
        if ((err = dev_alloc(m, (void**)&d_tiles, tl.size() * sizeof(int4))) != cudaSuccess) break;
        err = dev_upload(m, d_tiles, tl.data(), tl.size() * sizeof(int4));
        if (err == cudaSuccess) err = dev_sync(m);
        float ms = 0.0f;
        const int first = c == kCand[0] ? 0 : 1;  // one warm-up launch per element type
        for (int rep = first; rep < 3 && err == cudaSuccess; ++rep) {
          if ((err = cudaEventRecord(e0, s)) != cudaSuccess) break;
          if ((err = launch_apply2d_tiles(dt, m, L, d_tiles, int(tl.size()), x, y, s)) != cudaSuccess) break;
          if ((err = cudaEventRecord(e1, s)) != cudaSuccess) break;
          if ((err = cudaEventSynchronize(e1)) != cudaSuccess) break;
          float t = 0.0f;
          if ((err = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
          if (rep == 1 || (rep > 1 && t < ms)) ms = t;
        }
        const cudaError_t ef = cudaStreamSynchronize(s);
        dev_free(m, d_tiles);
        if (err == cudaSuccess) err = ef;
        if (err != cudaSuccess) break;
        if (best == 0 || ms < best_ms) {
          best = c;
          best_ms = ms;
        }
      }
      if (err != cudaSuccess) break;
      std::lock_guard<std::mutex> lk(mu);
      cache[key] = best;
    }
    const std::vector<int4> tl = tile_list_2d(L.n, best, kTileWidth2);
    if ((err = dev_alloc(m, (void**)&L.tiles_dt[dt], tl.size() * sizeof(int4))) != cudaSuccess) break;
    if ((err = dev_upload(m, L.tiles_dt[dt], tl.data(), tl.size() * sizeof(int4))) != cudaSuccess) break;
    L.n_tiles_dt[dt] = int(tl.size());
    L.tile_rows[dt] = best;
  }
  if (err == cudaSuccess) err = dev_sync(m);
  cleanup();
  return err;
}

}  // namespace hyteg
