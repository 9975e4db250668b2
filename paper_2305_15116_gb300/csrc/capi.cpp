// The C ABI of libhyteg.so (declared in include/hyteg.h): argument checks,
// error codes and the launch sequence of one operator apply.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/hyteg.h"
#include "hyteg_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(HYTEG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

using hyteg::check_level;
using hyteg::elem_size;
using hyteg::valid_dtype;

// Host-only queries need no refined device tables.
int check_host_level(const hyteg_mesh* mesh, int level) {
  if (!mesh) return fail(HYTEG_EINVAL, "mesh is NULL");
  if (level < 0 || level > 15) return fail(HYTEG_EINVAL, "level must be in 0..15");
  return HYTEG_OK;
}

}  // namespace

void hyteg::set_last_error(const std::string& msg) { g_last_error = msg; }

size_t hyteg::elem_size(int dtype) { return dtype == HYTEG_F32 ? 4 : 8; }

bool hyteg::valid_dtype(int dtype) { return dtype == HYTEG_F64 || dtype == HYTEG_F32 || dtype == HYTEG_F64_IEEE; }

int hyteg::check_level(const hyteg_mesh* mesh, int level) {
  if (!mesh) return fail(HYTEG_EINVAL, "mesh is NULL");
  if (level < 0) return fail(HYTEG_EINVAL, "level < 0");
  if (level > mesh->m.max_level)
    return fail(HYTEG_ESTATE, "level " + std::to_string(level) + " not refined (max " +
                                  std::to_string(mesh->m.max_level) + ")");
  return HYTEG_OK;
}

extern "C" {

int hyteg_mesh_create(int dim, int64_t n_verts, const double* coords, int64_t n_cells, const int64_t* cells,
                      int bc, hyteg_mesh** out) {
  if (!out) return fail(HYTEG_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return fail(HYTEG_EINVAL, "dim must be 2 or 3");
  if (n_verts < dim + 1 || n_cells < 1) return fail(HYTEG_EINVAL, "too few vertices or cells");
  if (n_cells > (int64_t(1) << 30) || n_verts > (int64_t(1) << 30)) return fail(HYTEG_EINVAL, "mesh too large");
  if (!coords || !cells) return fail(HYTEG_EINVAL, "coords or cells is NULL");
  if (bc != HYTEG_BC_NONE && bc != HYTEG_BC_DIRICHLET) return fail(HYTEG_EINVAL, "unknown bc");
  hyteg_mesh* h = new (std::nothrow) hyteg_mesh();
  if (!h) return fail(HYTEG_ENOMEM, "host allocation failed");
  try {
    h->m.dim = dim;
    h->m.bc = bc;
    h->m.n_verts = n_verts;
    h->m.n_cells = n_cells;
    h->m.coords.assign(coords, coords + n_verts * dim);
    h->m.cells.assign(cells, cells + n_cells * (dim + 1));
    const std::string err = hyteg::build_topology(h->m);
    if (!err.empty()) {
      delete h;
      return fail(HYTEG_EMESH, err);
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(HYTEG_ENOMEM, "host allocation failed");
  }
  *out = h;
  return HYTEG_OK;
}

int hyteg_mesh_refine(hyteg_mesh* mesh, int max_level) {
  if (!mesh) return fail(HYTEG_EINVAL, "mesh is NULL");
  if (max_level < 0 || max_level > 15) return fail(HYTEG_EINVAL, "max_level must be in 0..15");
  hyteg::Mesh& m = mesh->m;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (m.device >= 0 && m.device != dev) return fail(HYTEG_ESTATE, "refine called on a different device");
  try {
    if (!m.d_prims) {
      m.device = dev;  // from here on destroy releases what was allocated
      e = hyteg::dev_alloc(m, (void**)&m.d_prims, m.prims.size() * sizeof(hyteg::Prim));
      if (e != cudaSuccess) return fail(HYTEG_ENOMEM, "device allocation failed");
      e = hyteg::dev_upload(m, m.d_prims, m.prims.data(), m.prims.size() * sizeof(hyteg::Prim));
      if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
      e = hyteg::dev_alloc(m, (void**)&m.d_incs, m.incs.size() * sizeof(hyteg::Inc));
      if (e != cudaSuccess) return fail(HYTEG_ENOMEM, "device allocation failed");
      e = hyteg::dev_upload(m, m.d_incs, m.incs.data(), m.incs.size() * sizeof(hyteg::Inc));
      if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    }
    for (int l = m.max_level + 1; l <= max_level; ++l) {
      hyteg::LevelDev L;
      const std::string err = hyteg::build_level(m, l, L);
      if (!err.empty()) {
        hyteg::free_level(m, L);
        return fail(err.rfind("device allocation", 0) == 0 ? HYTEG_ENOMEM : HYTEG_ECUDA, err);
      }
      m.levels.push_back(L);
      m.max_level = l;
      if (m.dim == 3) {  // pick the 3D slab kernel's work split for this level
        e = hyteg::slab3d_autotune(m, m.levels.back());
        if (e != cudaSuccess) return cuda_fail(e, "slab work-split autotuning");
      } else {  // and the 2D kernel's tile height
        e = hyteg::tiles2d_autotune(m, m.levels.back());
        if (e != cudaSuccess) return cuda_fail(e, "2D tile autotuning");
      }
    }
    e = hyteg::dev_sync(m);
    if (e != cudaSuccess) return cuda_fail(e, "refine");
  } catch (const std::bad_alloc&) {
    return fail(HYTEG_ENOMEM, "host allocation failed");
  }
  return HYTEG_OK;
}

void hyteg_mesh_destroy(hyteg_mesh* mesh) {
  if (!mesh) return;
  hyteg::Mesh& m = mesh->m;
  if (m.device >= 0) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(m.device);
    if (m.mem.arena)
      hyteg::dev_sync(m);
    else
      cudaDeviceSynchronize();
    for (auto& L : m.levels) hyteg::free_level(m, L);
    hyteg::dev_free(m, m.d_prims);
    hyteg::dev_free(m, m.d_incs);
    cudaFree(m.stage_x);
    cudaFree(m.stage_y);
    hyteg::solver_free(m);
    hyteg::problem_free(m);
    cudaSetDevice(cur);
  }
  delete mesh;
}

int hyteg_autotune_choice(const hyteg_mesh* mesh, int level, int dtype, int* value) {
  if (int r = check_level(mesh, level)) return r;
  if (!value) return fail(HYTEG_EINVAL, "value is NULL");
  if (dtype != HYTEG_F64 && dtype != HYTEG_F32 && dtype != HYTEG_F64_IEEE) return fail(HYTEG_EINVAL, "bad dtype");
  const hyteg::LevelDev& L = mesh->m.levels[level];
  *value = mesh->m.dim == 3 ? L.slab_chunks[dtype] : L.tile_rows[dtype];
  return HYTEG_OK;
}

int hyteg_num_slots(const hyteg_mesh* mesh, int level, int64_t* n_slots, int64_t* n_global) {
  if (int r = check_host_level(mesh, level)) return r;
  if (n_slots) *n_slots = mesh->m.n_cells * hyteg::slots_per_macro(mesh->m.dim, level);
  if (n_global) *n_global = hyteg::n_global_dofs(mesh->m, level);
  return HYTEG_OK;
}

int hyteg_dof_map(const hyteg_mesh* mesh, int level, int64_t* global_id) {
  if (int r = check_host_level(mesh, level)) return r;
  if (!global_id) return fail(HYTEG_EINVAL, "global_id is NULL");
  try {
    hyteg::compute_dof_map(mesh->m, level, global_id);
  } catch (const std::exception& ex) {
    return fail(HYTEG_EINVAL, ex.what());
  }
  return HYTEG_OK;
}

int hyteg_apply_timed(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream,
                      void* ev_begin, void* ev_mid, void* ev_end) {
  if (int r = check_level(mesh, level)) return r;
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (!x || !y) return fail(HYTEG_EINVAL, "x or y is NULL");
  const hyteg::Mesh& m = mesh->m;
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, level)) * elem_size(dtype);
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  if (xb < yb + bytes && yb < xb + bytes) return fail(HYTEG_EINVAL, "x and y overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (ev_begin && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_begin), s)) != cudaSuccess)
    return cuda_fail(e, "cudaEventRecord");
  const char* what = "";
  e = hyteg::launch_apply(m, level, dtype, x, y, s, static_cast<cudaEvent_t>(ev_mid), &what);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (ev_end && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_end), s)) != cudaSuccess)
    return cuda_fail(e, "cudaEventRecord");
  return HYTEG_OK;
}

int hyteg_apply(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream) {
  return hyteg_apply_timed(mesh, level, dtype, x, y, stream, nullptr, nullptr, nullptr);
}

int hyteg_apply_partial(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream) {
  if (int r = check_level(mesh, level)) return r;
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (!x || !y) return fail(HYTEG_EINVAL, "x or y is NULL");
  const hyteg::Mesh& m = mesh->m;
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, level)) * elem_size(dtype);
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  if (xb < yb + bytes && yb < xb + bytes) return fail(HYTEG_EINVAL, "x and y overlap");
  const char* what = "";
  const cudaError_t e = hyteg::launch_apply_partial(m, level, dtype, x, y, static_cast<cudaStream_t>(stream), &what);
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, what);
}

int hyteg_apply_batch(const hyteg_mesh* const* meshes, const int* levels, int dtype, const void* const* xs,
                      void* const* ys, int count, void* stream) {
  if (count < 0) return fail(HYTEG_EINVAL, "count < 0");
  if (count == 0) return HYTEG_OK;
  if (!meshes || !levels || !xs || !ys) return fail(HYTEG_EINVAL, "NULL array");
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  // validate everything before the first launch
  for (int i = 0; i < count; ++i) {
    if (int r = check_level(meshes[i], levels[i])) return r;
    if (!xs[i] || !ys[i]) return fail(HYTEG_EINVAL, "x or y is NULL (entry " + std::to_string(i) + ")");
    const hyteg::Mesh& m = meshes[i]->m;
    const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, levels[i])) * elem_size(dtype);
    const char* xb = static_cast<const char*>(xs[i]);
    const char* yb = static_cast<const char*>(ys[i]);
    if (xb < yb + bytes && yb < xb + bytes)
      return fail(HYTEG_EINVAL, "x and y overlap (entry " + std::to_string(i) + ")");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const hyteg::Mesh*> m2;
  std::vector<int> l2;
  std::vector<const void*> x2;
  std::vector<void*> y2;
  for (int i = 0; i < count; ++i) {
    const hyteg::Mesh& m = meshes[i]->m;
    // 2D products share the batched launch, except float64 ones on a level
    // whose weights need the native fp64 kernel (outside the float-float range)
    if (m.dim == 2 && (dtype != HYTEG_F64 || m.levels[levels[i]].ff_ok)) {
      m2.push_back(&m);
      l2.push_back(levels[i]);
      x2.push_back(xs[i]);
      y2.push_back(ys[i]);
    } else {  // 3D meshes and the others: their own launches, in order
      const char* what = "";
      const cudaError_t e = hyteg::launch_apply(m, levels[i], dtype, xs[i], ys[i], s, nullptr, &what);
      if (e != cudaSuccess) return cuda_fail(e, what);
    }
  }
  if (!m2.empty()) {
    const cudaError_t e = hyteg::launch_apply2d_batch(dtype, m2.data(), l2.data(), x2.data(), y2.data(),
                                                      int(m2.size()), s);
    if (e != cudaSuccess) return cuda_fail(e, "batched 2D apply kernel");
  }
  return HYTEG_OK;
}

int hyteg_apply_host(hyteg_mesh* mesh, int level, int dtype, const void* x_host, void* y_host, void* stream) {
  if (int r = check_level(mesh, level)) return r;
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (!x_host || !y_host) return fail(HYTEG_EINVAL, "x_host or y_host is NULL");
  hyteg::Mesh& m = mesh->m;
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, level)) * elem_size(dtype);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (m.stage_bytes < bytes) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(m.stage_x);
    cudaFree(m.stage_y);
    m.stage_x = m.stage_y = nullptr;
    m.stage_bytes = 0;
    if (cudaMalloc(&m.stage_x, bytes) != cudaSuccess || cudaMalloc(&m.stage_y, bytes) != cudaSuccess) {
      cudaFree(m.stage_x);
      m.stage_x = nullptr;
      cudaGetLastError();
      return fail(HYTEG_ENOMEM, "device staging allocation failed");
    }
    m.stage_bytes = bytes;
  }
  e = cudaMemcpyAsync(m.stage_x, x_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
  if (int r = hyteg_apply(mesh, level, dtype, m.stage_x, m.stage_y, stream)) return r;
  e = cudaMemcpyAsync(y_host, m.stage_y, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return HYTEG_OK;
}

int hyteg_apply_host_batch(hyteg_mesh* mesh, int level, int dtype, const void* const* x_hosts,
                           void* const* y_hosts, int count, void* stream) {
  if (int r = check_level(mesh, level)) return r;
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (count < 0 || (count > 0 && (!x_hosts || !y_hosts))) return fail(HYTEG_EINVAL, "bad batch");
  for (int i = 0; i < count; ++i)
    if (!x_hosts[i] || !y_hosts[i]) return fail(HYTEG_EINVAL, "NULL host vector in the batch");
  if (count == 0) return HYTEG_OK;
  hyteg::Mesh& m = mesh->m;
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, level)) * elem_size(dtype);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // two staging pairs, one allocation each for x and y
  if (m.stage_bytes < 2 * bytes) {
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(m.stage_x);
    cudaFree(m.stage_y);
    m.stage_x = m.stage_y = nullptr;
    m.stage_bytes = 0;
    if (cudaMalloc(&m.stage_x, 2 * bytes) != cudaSuccess || cudaMalloc(&m.stage_y, 2 * bytes) != cudaSuccess) {
      cudaFree(m.stage_x);
      m.stage_x = nullptr;
      cudaGetLastError();
      return fail(HYTEG_ENOMEM, "device staging allocation failed");
    }
    m.stage_bytes = 2 * bytes;
  }
  char* sx[2] = {static_cast<char*>(m.stage_x), static_cast<char*>(m.stage_x) + bytes};
  char* sy[2] = {static_cast<char*>(m.stage_y), static_cast<char*>(m.stage_y) + bytes};
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_cmp[2] = {nullptr, nullptr}, ev_down[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;
  auto cleanup = [&]() {
    if (up) cudaStreamSynchronize(up);
    if (down) cudaStreamSynchronize(down);
    cudaStreamSynchronize(cs);
    for (int k = 0; k < 2; ++k) {
      if (ev_up[k]) cudaEventDestroy(ev_up[k]);
      if (ev_cmp[k]) cudaEventDestroy(ev_cmp[k]);
      if (ev_down[k]) cudaEventDestroy(ev_down[k]);
    }
    if (ev_start) cudaEventDestroy(ev_start);
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
  };
#define HB_TRY(call, what)           \
  do {                               \
    e = (call);                      \
    if (e != cudaSuccess) {          \
      cleanup();                     \
      return cuda_fail(e, what);     \
    }                                \
  } while (0)
  HB_TRY(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking), "cudaStreamCreate");
  HB_TRY(cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking), "cudaStreamCreate");
  for (int k = 0; k < 2; ++k) {
    HB_TRY(cudaEventCreateWithFlags(&ev_up[k], cudaEventDisableTiming), "cudaEventCreate");
    HB_TRY(cudaEventCreateWithFlags(&ev_cmp[k], cudaEventDisableTiming), "cudaEventCreate");
    HB_TRY(cudaEventCreateWithFlags(&ev_down[k], cudaEventDisableTiming), "cudaEventCreate");
  }
  // the copies start after the caller's earlier work on `stream`
  HB_TRY(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming), "cudaEventCreate");
  HB_TRY(cudaEventRecord(ev_start, cs), "cudaEventRecord");
  HB_TRY(cudaStreamWaitEvent(up, ev_start, 0), "cudaStreamWaitEvent");
  for (int i = 0; i < count; ++i) {
    const int k = i & 1;
    if (i >= 2) HB_TRY(cudaStreamWaitEvent(up, ev_cmp[k], 0), "cudaStreamWaitEvent");  // x slot free
    HB_TRY(cudaMemcpyAsync(sx[k], x_hosts[i], bytes, cudaMemcpyHostToDevice, up), "cudaMemcpyAsync H2D");
    HB_TRY(cudaEventRecord(ev_up[k], up), "cudaEventRecord");
    HB_TRY(cudaStreamWaitEvent(cs, ev_up[k], 0), "cudaStreamWaitEvent");
    if (i >= 2) HB_TRY(cudaStreamWaitEvent(cs, ev_down[k], 0), "cudaStreamWaitEvent");  // y slot free
    const char* what = "";
    e = hyteg::launch_apply(m, level, dtype, sx[k], sy[k], cs, nullptr, &what);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(e, what);
    }
    HB_TRY(cudaEventRecord(ev_cmp[k], cs), "cudaEventRecord");
    HB_TRY(cudaStreamWaitEvent(down, ev_cmp[k], 0), "cudaStreamWaitEvent");
    HB_TRY(cudaMemcpyAsync(y_hosts[i], sy[k], bytes, cudaMemcpyDeviceToHost, down), "cudaMemcpyAsync D2H");
    HB_TRY(cudaEventRecord(ev_down[k], down), "cudaEventRecord");
  }
#undef HB_TRY
  e = cudaStreamSynchronize(down);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return HYTEG_OK;
}

int hyteg_slot_coords(const hyteg_mesh* mesh, int level, double* xyz) {
  if (int r = check_host_level(mesh, level)) return r;
  if (!xyz) return fail(HYTEG_EINVAL, "xyz is NULL");
  hyteg::compute_slot_coords(mesh->m, level, xyz);
  return HYTEG_OK;
}

int hyteg_lumped_mass(const hyteg_mesh* mesh, int level, double* mass) {
  if (int r = check_host_level(mesh, level)) return r;
  if (!mass) return fail(HYTEG_EINVAL, "mass is NULL");
  hyteg::compute_lumped_mass(mesh->m, level, mass);
  return HYTEG_OK;
}

int hyteg_dirichlet_mask(const hyteg_mesh* mesh, int level, uint8_t* mask) {
  if (int r = check_host_level(mesh, level)) return r;
  if (!mask) return fail(HYTEG_EINVAL, "mask is NULL");
  hyteg::compute_dirichlet_mask(mesh->m, level, mask);
  return HYTEG_OK;
}

int hyteg_solver_setup(hyteg_mesh* mesh, int max_level, int nu1, int nu2, double omega) {
  if (int r = check_level(mesh, max_level)) return r;
  if (nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || nu1 > 64 || nu2 > 64) return fail(HYTEG_EINVAL, "bad sweep counts");
  if (!(omega > 0.0 && omega < 2.0)) return fail(HYTEG_EINVAL, "omega must lie in (0, 2)");
  if (mesh->m.bc != HYTEG_BC_DIRICHLET) return fail(HYTEG_EINVAL, "the solver needs Dirichlet boundary rows");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != mesh->m.device) return fail(HYTEG_ESTATE, "current device is not the mesh's device");
  try {
    const std::string err = hyteg::solver_setup(mesh->m, max_level, nu1, nu2, omega);
    if (!err.empty()) {
      hyteg::solver_free(mesh->m);
      const int code = err.find("device allocation") != std::string::npos ? HYTEG_ENOMEM
                       : err.rfind("cuda", 0) == 0                         ? HYTEG_ECUDA
                                                                           : HYTEG_EINVAL;
      return fail(code, err);
    }
  } catch (const std::bad_alloc&) {
    hyteg::solver_free(mesh->m);
    return fail(HYTEG_ENOMEM, "host allocation failed");
  }
  return HYTEG_OK;
}

namespace {
int check_solver(const hyteg_mesh* mesh, int level, int min_level) {
  if (int r = check_level(mesh, level)) return r;
  if (!mesh->m.solver || level > mesh->m.solver->max_level)
    return fail(HYTEG_ESTATE, "hyteg_solver_setup has not covered this level");
  if (level < min_level) return fail(HYTEG_EINVAL, "level too small for this operation");
  return HYTEG_OK;
}
}  // namespace

int hyteg_restrict(const hyteg_mesh* mesh, int fine_level, int dtype, const void* r_fine, void* b_coarse,
                   void* stream) {
  if (int r = check_solver(mesh, fine_level, 1)) return r;
  if (dtype != HYTEG_F64 && dtype != HYTEG_F32) return fail(HYTEG_EINVAL, "dtype must be HYTEG_F64 or HYTEG_F32");
  if (!r_fine || !b_coarse) return fail(HYTEG_EINVAL, "NULL vector");
  const cudaError_t e =
      hyteg::mg_restrict(mesh->m, fine_level, dtype, r_fine, b_coarse, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "restriction");
}

int hyteg_prolong_add(const hyteg_mesh* mesh, int fine_level, int dtype, const void* e_coarse, void* u_fine,
                      void* stream) {
  if (int r = check_solver(mesh, fine_level, 1)) return r;
  if (dtype != HYTEG_F64 && dtype != HYTEG_F32) return fail(HYTEG_EINVAL, "dtype must be HYTEG_F64 or HYTEG_F32");
  if (!e_coarse || !u_fine) return fail(HYTEG_EINVAL, "NULL vector");
  const cudaError_t e =
      hyteg::mg_prolong_add(mesh->m, fine_level, dtype, e_coarse, u_fine, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "prolongation");
}

int hyteg_vcycle(hyteg_mesh* mesh, int level, int dtype, const void* b, void* u, void* stream) {
  if (int r = check_solver(mesh, level, 0)) return r;
  if (dtype != HYTEG_F64 && dtype != HYTEG_F32) return fail(HYTEG_EINVAL, "dtype must be HYTEG_F64 or HYTEG_F32");
  if (!b || !u) return fail(HYTEG_EINVAL, "NULL vector");
  const cudaError_t e = hyteg::mg_vcycle(mesh->m, level, dtype, b, u, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "V-cycle");
}

int hyteg_solve(hyteg_mesh* mesh, int level, int mode, const double* b, double* u, double rtol, int max_iter,
                void* stream, int* iters, double* relres) {
  if (int r = check_solver(mesh, level, 0)) return r;
  if (mode != HYTEG_SOLVE_F64 && mode != HYTEG_SOLVE_MIXED) return fail(HYTEG_EINVAL, "unknown mode");
  if (!b || !u || !iters || !relres) return fail(HYTEG_EINVAL, "NULL argument");
  if (!(rtol > 0.0) || max_iter < 0) return fail(HYTEG_EINVAL, "bad rtol or max_iter");
  const cudaError_t e = hyteg::mg_solve(mesh->m, level, mode, b, u, nullptr, rtol, max_iter,
                                        static_cast<cudaStream_t>(stream), iters, relres);
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "solve");
}

int hyteg_solve_two_part(hyteg_mesh* mesh, int level, int mode, const double* b, double* u, double* u_lo,
                         double rtol, int max_iter, void* stream, int* iters, double* relres) {
  if (int r = check_solver(mesh, level, 0)) return r;
  if (mode != HYTEG_SOLVE_F64 && mode != HYTEG_SOLVE_MIXED) return fail(HYTEG_EINVAL, "unknown mode");
  if (!b || !u || !u_lo || !iters || !relres) return fail(HYTEG_EINVAL, "NULL argument");
  if (u_lo == u) return fail(HYTEG_EINVAL, "u and u_lo must be different vectors");
  if (!(rtol > 0.0) || max_iter < 0) return fail(HYTEG_EINVAL, "bad rtol or max_iter");
  const cudaError_t e = hyteg::mg_solve(mesh->m, level, mode, b, u, u_lo, rtol, max_iter,
                                        static_cast<cudaStream_t>(stream), iters, relres);
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "solve");
}

int hyteg_solve_two_part_group(hyteg_mesh* const* meshes, int count, int level, int mode, const double* const* b,
                               double* const* u, double* const* u_lo, double rtol, int max_iter, void* stream,
                               int* iters, double* relres) {
  if (count < 1) return fail(HYTEG_EINVAL, "count < 1");
  if (!meshes || !b || !u || !u_lo || !iters || !relres) return fail(HYTEG_EINVAL, "NULL argument");
  if (mode != HYTEG_SOLVE_F64 && mode != HYTEG_SOLVE_MIXED) return fail(HYTEG_EINVAL, "unknown mode");
  if (!(rtol > 0.0) || max_iter < 0) return fail(HYTEG_EINVAL, "bad rtol or max_iter");
  std::vector<hyteg::Mesh*> ms(count);
  for (int i = 0; i < count; ++i) {
    if (int r = check_solver(meshes[i], level, 0)) return r;
    const std::string at = " (entry " + std::to_string(i) + ")";
    if (!b[i] || !u[i] || !u_lo[i]) return fail(HYTEG_EINVAL, "NULL vector" + at);
    if (u_lo[i] == u[i]) return fail(HYTEG_EINVAL, "u and u_lo must be different vectors" + at);
    ms[i] = &meshes[i]->m;
    if (ms[i]->dim != ms[0]->dim) return fail(HYTEG_EINVAL, "meshes of different dimensions" + at);
    if (ms[i]->solver->nu1 != ms[0]->solver->nu1 || ms[i]->solver->nu2 != ms[0]->solver->nu2)
      return fail(HYTEG_EINVAL, "meshes with different sweep counts" + at);
    for (int j = 0; j < i; ++j)
      if (ms[j] == ms[i]) return fail(HYTEG_EINVAL, "a mesh appears twice" + at);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // 3D levels above the slab kernel's (n > 64) have no group launch: the
  // meshes are solved one after another
  if (ms[0]->dim == 3 && ms[0]->levels[level].n_slabs == 0) {
    for (int i = 0; i < count; ++i) {
      const cudaError_t e = hyteg::mg_solve(*ms[i], level, mode, b[i], u[i], u_lo[i], rtol, max_iter, s, iters + i,
                                            relres + i);
      if (e != cudaSuccess) return cuda_fail(e, "solve");
    }
    return HYTEG_OK;
  }
  const cudaError_t e = hyteg::mg_solve_group(ms.data(), count, level, mode, b, u, u_lo, rtol, max_iter, s, iters,
                                              relres);
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "group solve");
}

int hyteg_p2_num_slots(const hyteg_mesh* mesh, int level, int64_t* n_slots, int64_t* n_global) {
  if (int r = check_host_level(mesh, level)) return r;
  if (mesh->m.dim != 2) return fail(HYTEG_EINVAL, "the P2 operator is built for 2D meshes");
  if (n_slots) *n_slots = mesh->m.n_cells * hyteg::p2_slots_per_macro(level);
  if (n_global) *n_global = hyteg::p2_n_global(mesh->m, level);
  return HYTEG_OK;
}

int hyteg_p2_dof_map(const hyteg_mesh* mesh, int level, int64_t* global_id) {
  if (int r = check_host_level(mesh, level)) return r;
  if (mesh->m.dim != 2) return fail(HYTEG_EINVAL, "the P2 operator is built for 2D meshes");
  if (!global_id) return fail(HYTEG_EINVAL, "global_id is NULL");
  try {
    hyteg::compute_p2_dof_map(mesh->m, level, global_id);
  } catch (const std::exception& ex) {
    return fail(HYTEG_EINVAL, ex.what());
  }
  return HYTEG_OK;
}

int hyteg_p2_apply_timed(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream,
                         void* ev_begin, void* ev_mid, void* ev_end) {
  if (int r = check_level(mesh, level)) return r;
  if (mesh->m.dim != 2) return fail(HYTEG_EINVAL, "the P2 operator is built for 2D meshes");
  if (!valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (!x || !y) return fail(HYTEG_EINVAL, "x or y is NULL");
  const hyteg::Mesh& m = mesh->m;
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::p2_slots_per_macro(level)) * elem_size(dtype);
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  if (xb < yb + bytes && yb < xb + bytes) return fail(HYTEG_EINVAL, "x and y overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (ev_begin && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_begin), s)) != cudaSuccess)
    return cuda_fail(e, "cudaEventRecord");
  const char* what = "";
  e = hyteg::launch_p2_apply(m, level, dtype, x, y, s, static_cast<cudaEvent_t>(ev_mid), &what);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (ev_end && (e = cudaEventRecord(static_cast<cudaEvent_t>(ev_end), s)) != cudaSuccess)
    return cuda_fail(e, "cudaEventRecord");
  return HYTEG_OK;
}

int hyteg_p2_apply(const hyteg_mesh* mesh, int level, int dtype, const void* x, void* y, void* stream) {
  return hyteg_p2_apply_timed(mesh, level, dtype, x, y, stream, nullptr, nullptr, nullptr);
}

int hyteg_poisson_rhs(hyteg_mesh* mesh, int level, uint64_t seed, double noise, double* b, void* stream) {
  if (int r = check_solver(mesh, level, 0)) return r;
  if (!b) return fail(HYTEG_EINVAL, "b is NULL");
  if (!(noise >= 0.0) || !std::isfinite(noise)) return fail(HYTEG_EINVAL, "noise must be finite and >= 0");
  hyteg::Mesh& m = mesh->m;
  if (!m.problem.ready) {
    const std::string err = hyteg::problem_setup(m);
    if (!err.empty()) {
      hyteg::problem_free(m);
      return fail(err.find("allocation") != std::string::npos ? HYTEG_ENOMEM : HYTEG_ECUDA, err);
    }
  }
  const cudaError_t e = hyteg::poisson_rhs(m, level, seed, noise, b, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "right-hand side");
}

int hyteg_to_global(const hyteg_mesh* mesh, int level, const double* v, double* v_global, void* stream) {
  if (int r = check_solver(mesh, level, 0)) return r;
  if (!v || !v_global) return fail(HYTEG_EINVAL, "NULL vector");
  const cudaError_t e = hyteg::to_global(mesh->m, level, v, v_global, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HYTEG_OK : cuda_fail(e, "global gather");
}

const char* hyteg_last_error(void) { return g_last_error.c_str(); }

const char* hyteg_version(void) { return "hyteg-gb300 0.1 (sm_103a)"; }

}  // extern "C"
