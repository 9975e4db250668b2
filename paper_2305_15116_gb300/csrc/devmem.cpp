// Device memory of a mesh: plain cudaMalloc, or blocks of an arena.
//
// A mesh created through the C ABI allocates with cudaMalloc.  A mesh owned by
// the solve server allocates from the server's arena: one device region
// reserved up front and split with a first-fit free list on the host, so that
// building and dropping cached meshes neither calls cudaMalloc nor cudaFree
// (cudaFree synchronises the whole device, which would stall every request in
// flight) and the server's memory cap is a hard limit.
#include <map>
#include <mutex>
#include <unordered_map>

#include "hyteg_internal.h"

namespace hyteg {

struct Arena {
  char* base = nullptr;
  size_t size = 0;
  size_t used = 0;
  std::map<size_t, size_t> free_blocks;            // offset -> size, coalesced
  std::unordered_map<size_t, size_t> live;         // offset -> size
  int fail_next = 0;                               // injected failures still to come
  std::mutex mu;
};

namespace {
constexpr size_t kAlign = 256;
size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }
}  // namespace

Arena* arena_create(size_t bytes, std::string& err) {
  Arena* a = new Arena();
  a->size = round_up(bytes);
  const cudaError_t e = cudaMalloc((void**)&a->base, a->size);
  if (e != cudaSuccess) {
    err = std::string("cudaMalloc of the arena: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete a;
    return nullptr;
  }
  a->free_blocks[0] = a->size;
  return a;
}

void arena_destroy(Arena* a) {
  if (!a) return;
  cudaFree(a->base);
  delete a;
}

void* arena_alloc(Arena* a, size_t bytes) {
  const size_t need = round_up(bytes ? bytes : 1);
  std::lock_guard<std::mutex> lk(a->mu);
  if (a->fail_next > 0) {  // a failure injected on the host (testing the failure paths)
    --a->fail_next;
    return nullptr;
  }
  for (auto it = a->free_blocks.begin(); it != a->free_blocks.end(); ++it) {
    if (it->second < need) continue;
    const size_t off = it->first, sz = it->second;
    a->free_blocks.erase(it);
    if (sz > need) a->free_blocks[off + need] = sz - need;
    a->live[off] = need;
    a->used += need;
    return a->base + off;
  }
  return nullptr;
}

void arena_inject_failures(Arena* a, int count) {
  std::lock_guard<std::mutex> lk(a->mu);
  a->fail_next = count > 0 ? count : 0;
}

void arena_free(Arena* a, void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(a->mu);
  const size_t off = size_t(static_cast<char*>(p) - a->base);
  auto lv = a->live.find(off);
  if (lv == a->live.end()) return;  // not ours: ignore
  size_t start = off, sz = lv->second;
  a->live.erase(lv);
  a->used -= sz;
  auto next = a->free_blocks.lower_bound(start);
  if (next != a->free_blocks.end() && next->first == start + sz) {
    sz += next->second;
    next = a->free_blocks.erase(next);
  }
  if (next != a->free_blocks.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      sz += prev->second;
      a->free_blocks.erase(prev);
    }
  }
  a->free_blocks[start] = sz;
}

size_t arena_used(Arena* a) {
  std::lock_guard<std::mutex> lk(a->mu);
  return a->used;
}

size_t arena_free_bytes(Arena* a) {
  std::lock_guard<std::mutex> lk(a->mu);
  return a->size - a->used;
}

size_t arena_largest_free(Arena* a) {
  std::lock_guard<std::mutex> lk(a->mu);
  size_t best = 0;
  for (const auto& kv : a->free_blocks) best = kv.second > best ? kv.second : best;
  return best;
}

cudaError_t dev_alloc(const Mesh& m, void** p, size_t bytes) {
  if (m.mem.region) {
    DevMem& mm = const_cast<DevMem&>(m.mem);
    const size_t need = round_up(bytes ? bytes : 1);
    if (mm.region_used + need <= mm.region_size) {
      *p = mm.region + mm.region_used;
      mm.region_used += need;
      return cudaSuccess;
    }
  }
  if (m.mem.arena) {
    *p = arena_alloc(m.mem.arena, bytes);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes ? bytes : 1);
}

void dev_free(const Mesh& m, void* p) {
  if (!p) return;
  if (m.mem.region && static_cast<char*>(p) >= m.mem.region && static_cast<char*>(p) < m.mem.region + m.mem.region_size)
    return;  // released with the region
  if (m.mem.arena) {
    // Arena blocks are handed to the next allocation at once, possibly on
    // another stream: drain the work this mesh queued (uploads, clears,
    // kernels) first, so that nothing of it lands in the block's next owner.
    cudaStreamSynchronize(m.mem.stream);
    arena_free(m.mem.arena, p);
  } else {
    cudaFree(p);  // synchronises the device itself
  }
}

cudaError_t dev_upload(const Mesh& m, void* dst, const void* src, size_t bytes) {
  if (!bytes) return cudaSuccess;
  // pageable source: the call returns once the source has been consumed
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, m.mem.stream);
}

cudaError_t dev_zero(const Mesh& m, void* p, size_t bytes) {
  if (!bytes) return cudaSuccess;
  return cudaMemsetAsync(p, 0, bytes, m.mem.stream);
}

cudaError_t dev_sync(const Mesh& m) { return cudaStreamSynchronize(m.mem.stream); }

}  // namespace hyteg
