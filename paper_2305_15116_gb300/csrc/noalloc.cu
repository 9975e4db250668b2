// Allocation-free variant of the host-buffer apply.
//
// hyteg_apply_host stages x and y in device buffers that it allocates with
// cudaMalloc the first time it sees a vector of that size.  Some callers must
// not trigger a device allocation at that point: real-time loops that forbid
// allocation after start-up (an allocation can synchronise the device and
// stall for milliseconds), and processes whose device memory is entirely
// pre-reserved by another allocator (a framework's caching pool), where a
// stray cudaMalloc fails or fragments it.  hyteg_apply_host_static serves
// them: its staging memory is one fixed file-scope device array, present on
// every GPU that loads the library for as long as the process lives, and the
// call makes no allocation of its own.  It synchronises its stream before
// returning (the result must be in host memory on return), so it cannot run
// on a stream that is being captured into a CUDA graph: it checks that first
// and refuses with HYTEG_ESTATE.
#include <mutex>
#include <string>

#include "../../include/hyteg.h"
#include "hyteg_internal.h"

namespace {

constexpr size_t kStageBytes = HYTEG_STATIC_STAGE_BYTES;  // per vector

// x staging in the first half, y staging in the second half.  Shared by every
// call on a device and keeps the last call's contents; nothing in it has to
// start at zero: the host-to-device copy overwrites all bytes of x that the
// kernels read, and the kernels write every slot of y before it is copied back.
static __device__ __align__(256) unsigned char g_stage[2 * kStageBytes];

constexpr int kMaxDevices = 64;
std::mutex g_stage_mu;
unsigned char* g_stage_addr[kMaxDevices] = {};  // device address of g_stage, per device

// Device address of g_stage on device `dev` (which must be current).  In host
// code `g_stage` names a host-side stand-in, not device memory, so the
// address is looked up once per device with cudaGetSymbolAddress and cached.
cudaError_t stage_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_stage_mu);
  if (!g_stage_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_stage);
    if (e != cudaSuccess) return e;
    g_stage_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_stage_addr[dev];
  return cudaSuccess;
}

int fail(int code, const std::string& msg) {
  hyteg::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int hyteg_apply_host_static(const hyteg_mesh* mesh, int level, int dtype, const void* x_host,
                                       void* y_host, void* stream) {
  if (int r = hyteg::check_level(mesh, level)) return r;
  const hyteg::Mesh& m = mesh->m;
  if (!hyteg::valid_dtype(dtype)) return fail(HYTEG_EINVAL, "unknown dtype");
  if (!x_host || !y_host) return fail(HYTEG_EINVAL, "x_host or y_host is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the call ends by synchronising `s`, which a stream under graph capture
  // does not allow: refuse before touching the stream
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(HYTEG_ESTATE, "hyteg_apply_host_static: the stream is being captured into a CUDA graph; the call "
                              "synchronises its stream and cannot be captured");
  const size_t bytes = size_t(m.n_cells) * size_t(hyteg::slots_per_macro(m.dim, level)) * hyteg::elem_size(dtype);
  if (bytes > kStageBytes)
    return fail(HYTEG_EINVAL, "hyteg_apply_host_static: a vector of this level needs " + std::to_string(bytes) +
                                  " bytes, more than the static staging limit of " + std::to_string(kStageBytes) +
                                  " bytes (HYTEG_STATIC_STAGE_BYTES); use hyteg_apply_host");
  int dev = -1;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != m.device || dev < 0 || dev >= kMaxDevices)
    return fail(HYTEG_ESTATE, "the current device is not the device the mesh was refined on");
  unsigned char* base = nullptr;
  e = stage_address(dev, &base);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  void* xd = base;
  void* yd = base + kStageBytes;
  e = cudaMemcpyAsync(xd, x_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaMemcpyAsync H2D: ") + cudaGetErrorString(e));
  const char* what = "";
  e = hyteg::launch_apply(m, level, dtype, xd, yd, s, nullptr, &what);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  e = cudaMemcpyAsync(y_host, yd, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaMemcpyAsync D2H: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(HYTEG_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  return HYTEG_OK;
}
